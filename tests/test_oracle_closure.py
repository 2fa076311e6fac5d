"""Pins of the oracle's M1 closure (Sec. 2, Eqs. (eddTens), (Udir)) and of
its HLL wave-speed table (Sec. 3.2) against limits and closed forms."""
import math

import numpy as np
import pytest

from oracle import hll_table as H


def test_chi_limits(oracle_mod):
    """Isotropic radiation (f = 0) has D = I/3; a beam (f = 1) keeps chi = 1."""
    assert oracle_mod.chi(0.0) == pytest.approx(1.0 / 3.0, abs=1e-16)
    assert oracle_mod.chi(1.0) == pytest.approx(1.0, abs=1e-16)
    fs = np.linspace(0, 1, 101)
    ch = [oracle_mod.chi(f) for f in fs]
    assert np.all(np.diff(ch) > 0)


def test_eddington_tensor_properties(oracle_mod):
    rng = np.random.default_rng(1)
    c = 3e9
    for _ in range(200):
        N = 10 ** rng.uniform(-5, 5)
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        f = rng.uniform(0, 1)
        D, fo, n = oracle_mod.eddington(c, N, f * c * N * d)
        assert np.trace(D) == pytest.approx(1.0, abs=1e-14)          # tr D = 1
        assert np.allclose(D, D.T, atol=0)
        assert fo == pytest.approx(f, rel=1e-12, abs=1e-15)
        # the flux direction is an eigenvector with eigenvalue chi
        assert np.allclose(D @ d, oracle_mod.chi(fo) * d, rtol=1e-12, atol=1e-14)
    D, f, _ = oracle_mod.eddington(c, 1.0, np.zeros(3))
    assert f == 0.0 and np.allclose(D, np.eye(3) / 3.0, atol=1e-16)
    D, f, _ = oracle_mod.eddington(c, 2.0, np.array([0.0, 0.0, 2.0 * c]))
    assert f == 1.0 and np.allclose(D, np.diag([0.0, 0.0, 1.0]), atol=1e-16)
    # f > 1 (unphysical input) is clamped
    D, f, _ = oracle_mod.eddington(c, 1.0, np.array([3.0 * c, 0.0, 0.0]))
    assert f == 1.0


def _one_d_eigs(f):
    """Closed form for mu = +1: the (N, F_x) block is the 1-D M1 system with
    Jacobian [[0, 1], [chi - f chi', chi']]; the transverse flux components
    move at (3 chi - 1) / (2 f)."""
    s = math.sqrt(4.0 - 3.0 * f * f)
    chi = (3.0 + 4.0 * f * f) / (5.0 + 2.0 * s)
    dchi = (8.0 * f * (5.0 + 2.0 * s) + (3.0 + 4.0 * f * f) * 6.0 * f / s) / (5.0 + 2.0 * s) ** 2
    disc = math.sqrt(dchi * dchi + 4.0 * (chi - f * dchi))
    l1 = 0.5 * (dchi - disc)
    l2 = 0.5 * (dchi + disc)
    lt = (3.0 * chi - 1.0) / (2.0 * f)
    return min(l1, l2, lt), max(l1, l2, lt)


def test_table_limits_and_symmetry():
    t = H.table()
    nf, nmu = t.shape[:2]
    r3 = 1.0 / math.sqrt(3.0)
    assert np.allclose(t[0, :, 0], -r3, atol=1e-15) and np.allclose(t[0, :, 1], r3, atol=1e-15)
    assert np.all(t[..., 0] <= t[..., 1])
    assert np.all(np.abs(t) <= 1.0 + 1e-12)                     # |lambda| <= c
    # lambda(f, -mu) = -reverse(lambda(f, mu))
    assert np.allclose(t[:, ::-1, 0], -t[:, :, 1], atol=1e-12)
    # mu = +1 column against the 1-D closed form
    for k in range(1, nf - 1):
        f = k / (nf - 1)
        lo, hi = _one_d_eigs(f)
        assert t[k, -1, 0] == pytest.approx(lo, abs=1e-12)
        assert t[k, -1, 1] == pytest.approx(hi, abs=1e-12)
    # beam limit f -> 1: all speeds collapse onto mu
    mus = -1.0 + 2.0 * np.arange(nmu) / (nmu - 1)
    assert np.max(np.abs(t[-2, :, 0] - mus)) < 0.15
    assert np.max(np.abs(t[-2, :, 1] - mus)) < 0.15


def test_lookup_interpolates(oracle_mod):
    t = H.table()
    lo, hi = oracle_mod.hll_lookup(t, 0.0, 0.3)
    assert lo == pytest.approx(-1 / math.sqrt(3)) and hi == pytest.approx(1 / math.sqrt(3))
    # on a grid node the lookup returns the node
    k, j = 100, 77
    f = k / 256.0
    mu = -1.0 + j / 128.0
    lo, hi = oracle_mod.hll_lookup(t, f, mu)
    assert lo == pytest.approx(t[k, j, 0], abs=1e-15) and hi == pytest.approx(t[k, j, 1], abs=1e-15)
    # between nodes the error against the exact eigenvalues is small
    for f, mu in [(0.3037, 0.1234), (0.77, -0.61), (0.51, 0.99)]:
        lo, hi = oracle_mod.hll_lookup(t, f, mu)
        elo, ehi = H.eigen_extremes(f, mu)
        assert abs(lo - elo) < 2e-4 and abs(hi - ehi) < 2e-4


def test_closure_floor(oracle_mod):
    """The closure-floor reading (Sec. 2, Eq. (Udir) gives f = |F|/(c N) and
    n = F/|F|, undefined for N = 0; the oracle takes f := 0, n := 0 for
    N <= 1e-30 photons/cm^3, the isotropic D = I/3).  Above the floor the
    closure is the printed one whatever the scale of N; at or below it a
    cell is isotropic whatever its F."""
    c = 3e9
    chi = lambda f: (3 + 4 * f * f) / (5 + 2 * np.sqrt(4 - 3 * f * f))  # noqa: E731
    d = np.array([0.6, -0.48, 0.64])
    for N in (2e-30, 1e-20, 1e-3, 1e4):
        F = 0.5 * c * N * d
        D, f, n = oracle_mod.eddington(c, N, F)
        assert f == pytest.approx(0.5, rel=1e-14)
        np.testing.assert_allclose(n, d, rtol=1e-14)
        a, b = 0.5 * (1 - chi(0.5)), 0.5 * (3 * chi(0.5) - 1)
        np.testing.assert_allclose(D, a * np.eye(3) + b * np.outer(d, d), rtol=1e-14, atol=1e-16)
    for N in (1e-30, 5e-31, 1e-300, 0.0):
        for scale in (0.5, 1.0, 1e10):   # the flux of such a cell does not matter
            D, f, n = oracle_mod.eddington(c, N, scale * c * max(N, 1e-30) * d)
            assert f == 0.0 and np.all(n == 0.0)
            np.testing.assert_allclose(D, np.eye(3) / 3.0, rtol=1e-15, atol=0.0)


def test_dark_cell_is_isotropic_in_hll(oracle_mod):
    """A cell at the floor gets the f = 0 wave speeds +-1/sqrt(3) in every
    direction, as an empty cell does."""
    from oracle import hll_table
    tab = hll_table.table()
    for N in (0.0, 1e-31):
        _, f, n = oracle_mod.eddington(3e9, N, np.array([1e-22, 0.0, 0.0]))
        for mu in n:
            lo, hi = oracle_mod.hll_lookup(tab, f, mu)
            assert lo == pytest.approx(-1 / np.sqrt(3), rel=1e-12)
            assert hi == pytest.approx(1 / np.sqrt(3), rel=1e-12)

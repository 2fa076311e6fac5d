"""Pins of the oracle's transport step (Sec. 3.2): photon conservation,
realisability, symmetry, and the exact free-streaming beam solution."""
import math

import numpy as np
import pytest
from scipy import stats

C = 2.99792458e10
SIG0 = np.zeros((1, 3))


def _problem(O, shape, flux, bc, G=1, cr=C / 100.0, dx=1e20):
    return O.Problem(shape, dx, G, cr, np.zeros((G, 3)), np.zeros((G, 3)), np.full(G, 3e-11),
                     X=1.0, isothermal=True, otsa=True, flux=flux, bc=bc, skip_thermo=True)


def _random_field(shape, G, cr, seed):
    rng = np.random.default_rng(seed)
    nc = int(np.prod(shape))
    N = 10 ** rng.uniform(-3, 0, size=(G, nc))
    d = rng.standard_normal((G, 3, nc))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    f = rng.uniform(0, 1, size=(G, 1, nc))
    F = cr * N[:, None, :] * f * d
    return N.reshape(-1).copy(), F.reshape(-1).copy()


@pytest.mark.parametrize("flux", [0, 1])
@pytest.mark.parametrize("bc,closed", [((0,) * 6, False), ((1,) * 6, True), ((2,) * 6, True),
                                       ((1, 0, 2, 2, 0, 1), False)])
def test_photon_conservation(oracle_mod, flux, bc, closed):
    """sum N V changes only by the net flux through the box faces
    (telescoping sum of Eq. (dUdt_sol)); closed boxes keep it exactly."""
    O = oracle_mod
    shape = (5, 6, 7)
    p = _problem(O, shape, flux, bc, G=2)
    s = O.new_state(shape, 2, 1e-3, 1e-6, 1e4)
    s["N"], s["F"] = _random_field(shape, 2, p.cfg.cr, 3)
    dt = O.courant_dt(0.8, p.cfg.dx, p.cfg.cr)
    V = p.cfg.dx ** 3
    for _ in range(3):
        before = s["N"].reshape(2, -1).sum(axis=1) * V
        st, b, _, _ = p.step(s, dt)
        after = s["N"].reshape(2, -1).sum(axis=1) * V
        assert st == 0
        assert np.allclose(b[:, 0], after, rtol=1e-15)
        for g in range(2):
            assert after[g] - before[g] == pytest.approx(-b[g, 2], abs=1e-13 * before[g])
            if closed:
                # zero up to the rounding of lambda(f, mu) vs lambda(f, -mu)
                assert abs(b[g, 2]) <= 1e-15 * before[g]
                assert after[g] == pytest.approx(before[g], rel=1e-14)


@pytest.mark.parametrize("flux", [0, 1])
def test_realisability_point_source(oracle_mod, flux):
    """|F| <= c_r N is kept by the explicit scheme at CFL 0.8."""
    O = oracle_mod
    shape = (9, 9, 9)
    p = _problem(O, shape, flux, (0,) * 6)
    s = O.new_state(shape, 1, 1e-3, 1e-6, 1e4)
    dt = O.courant_dt(0.8, p.cfg.dx, p.cfg.cr)
    for _ in range(25):
        p.step(s, dt, [[4, 4, 4]], [[1e50]])
    N = s["N"].reshape(-1)
    F = s["F"].reshape(3, -1)
    assert np.all(N >= 0)
    assert np.all(np.linalg.norm(F, axis=0) <= p.cfg.cr * N * (1 + 1e-13))
    assert np.any(np.linalg.norm(F, axis=0) > 0.5 * p.cfg.cr * N)   # radiation streams out


@pytest.mark.parametrize("flux", [0, 1])
def test_point_source_symmetry(oracle_mod, flux):
    """A centred isotropic source stays invariant under the 48 symmetries of
    the cube (axis permutations and reflections)."""
    O = oracle_mod
    n = 9
    p = _problem(O, (n, n, n), flux, (0,) * 6)
    s = O.new_state((n, n, n), 1, 1e-3, 1e-6, 1e4)
    dt = O.courant_dt(0.8, p.cfg.dx, p.cfg.cr)
    for _ in range(12):
        p.step(s, dt, [[4, 4, 4]], [[1e50]])
    N = s["N"].reshape(n, n, n)
    scale = N.max()
    for perm in [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]:
        Np = np.transpose(N, perm)
        assert np.max(np.abs(Np - N)) <= 1e-12 * scale
    for ax in range(3):
        assert np.max(np.abs(np.flip(N, ax) - N)) <= 1e-12 * scale
    Fx = s["F"].reshape(3, n, n, n)[0]
    assert np.max(np.abs(np.flip(Fx, 2) + Fx)) <= 1e-12 * p.cfg.cr * scale


@pytest.mark.parametrize("flux", [0, 1])
def test_free_streaming_beam_is_exact_upwind(oracle_mod, flux):
    """A plane beam with f = 1 along +x: both flux functions reduce to exact
    upwinding at Courant number nu = c dt/dx = CFL/3, whose solution for a
    step profile is N_i^n = N0 P(K >= i - i0), K ~ Binomial(n, nu); the
    beam stays at f = 1 (F = c N) behind and inside the front."""
    O = oracle_mod
    nx, i0 = 48, 9
    shape = (2, 2, nx)
    p = _problem(O, shape, flux, (0, 0, 2, 2, 2, 2))
    cr = p.cfg.cr
    s = O.new_state(shape, 1, 1e-3, 1e-6, 1e4)
    N0 = 2.5
    N = s["N"].reshape(shape)
    F = s["F"].reshape((3,) + shape)
    N[:, :, : i0 + 1] = N0
    F[0, :, :, : i0 + 1] = cr * N0
    dt = O.courant_dt(0.8, p.cfg.dx, cr)
    nu = cr * dt / p.cfg.dx
    assert nu == pytest.approx(0.8 / 3.0, rel=1e-15)
    nsteps = 60
    for _ in range(nsteps):
        p.step(s, dt)
    Nn = s["N"].reshape(shape)
    Fn = s["F"].reshape((3,) + shape)
    i = np.arange(nx)
    exact = N0 * stats.binom.sf(i - i0 - 1, nsteps, nu)
    for z in range(2):
        for y in range(2):
            assert np.max(np.abs(Nn[z, y] - exact)) <= 1e-12 * N0
            assert np.max(np.abs(Fn[0, z, y] - cr * Nn[z, y])) <= 1e-12 * cr * N0
    assert np.max(np.abs(Fn[1:])) <= 1e-12 * cr * N0
    # front (N = N0/2) moved by ~ c t
    front = i0 + 0.5 + nsteps * nu
    half = np.argmax(Nn[0, 0] < 0.5 * N0)
    assert abs(half - front) <= 1.5


def test_courant(oracle_mod):
    assert oracle_mod.courant_dt(0.8, 3.0, 1.0) == pytest.approx(0.8)

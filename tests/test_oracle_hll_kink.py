"""The HLL step is only piecewise differentiable: the intercell speeds are
max(0, lmax_L, lmax_R) and min(0, lmin_L, lmin_R) (Eq. (hll)), and where a
photon front runs into empty cells it gives them all the same F/N, so
neighbouring cells share (f, n) and their speeds tie exactly.  Along a
direction that moves such a cell the one-step map has a kink.

Pinned on the oracle (a 10^3 H+He box with two sources, three HLL steps
from neutral gas): along a random relative perturbation of every field the
forward and backward one-sided differences of a linear functional of the
next state differ by far more than rounding, at every step length; with
the photons of the cells returned by `parity.hll_tie_cells` left
unperturbed they agree to rounding, so the central difference is then the
derivative the adjoint is checked against.
"""
import numpy as np
import pytest

from parity import hll_tie_cells, oracle_problem


@pytest.fixture(scope="module")
def case(oracle_mod):
    from paper_1304_7126_gb300 import workloads as W
    O = oracle_mod
    w = W.small_cosmo(10, seed=3, nsrc=2, flux=O.HLL)
    p = oracle_problem(O, w, nthreads=4)
    dt = O.courant_dt(w.cfl, w.dx, w.cr)
    s0 = w.state()
    for _ in range(3):
        assert p.step(s0, dt, w.src_ijk, w.src_L)[0] == 0
    nc, G = w.ncells, w.G
    rng = np.random.default_rng(7)
    v = {"xHII": rng.standard_normal(nc), "T": rng.standard_normal(nc) / 1e4,
         "N": rng.standard_normal(G * nc) / s0["N"].max(),
         "F": rng.standard_normal(3 * G * nc) / (w.cr * s0["N"].max())}
    u = {"N": s0["N"] * rng.standard_normal(G * nc), "F": s0["F"] * rng.standard_normal(3 * G * nc) * 0.1,
         "T": s0["T"] * rng.standard_normal(nc)}

    def slopes(u, eps):
        def J(e):
            s = {k: a.copy() for k, a in s0.items()}
            for k, du in u.items():
                s[k] = s[k] + e * du
            st, _, sub, _ = p.step(s, dt, w.src_ijk, w.src_L)
            assert st == 0
            return sum(float(v[k] @ s[k]) for k in v), sub
        (jp, sp), (j0, s_), (jm, sm) = J(eps), J(0.0), J(-eps)
        assert np.array_equal(sp, s_) and np.array_equal(sm, s_)
        return (jp - j0) / eps, (j0 - jm) / eps

    return w, s0, u, slopes


def test_kink_at_tied_speeds(oracle_mod, case):
    w, s0, u, slopes = case
    for eps in (1e-6, 1e-8):
        fwd, bwd = slopes(u, eps)
        assert abs(fwd - bwd) > 1e-4 * abs(fwd), (eps, fwd, bwd)


def test_smooth_off_tied_cells(oracle_mod, case):
    w, s0, u, slopes = case
    tie = hll_tie_cells(oracle_mod, w, s0)
    assert 0 < tie.sum() < w.ncells // 20
    nc = w.ncells
    um = {k: (a * np.tile(~tie, a.size // nc) if k in ("N", "F") else a) for k, a in u.items()}
    fwd, bwd = slopes(um, 1e-7)
    assert abs(fwd - bwd) <= 1e-6 * abs(fwd), (fwd, bwd)

"""Pins of the oracle's smoothed RT (Sec. 3.4): the transport and injection
change of an RT step enters the thermochemistry as the rates
Ndot = (N' - N^t)/dt, Fdot = (F' - F^t)/dt (Eqs. (smoothrate1),
(smoothrate2)) of the semi-implicit photon update (App. A, Eq. (SIE
photons)), starting from the state before injection.

* Without absorption the smoothed step ends on the photon density and flux
  of the transport and injection steps (the paper's own limit statement).
* The photon ledger closes as without smoothing.
* With constant rates the update N_{k+1} = (N_k + h Ndot)/(1 + h D) has the
  fixed point Ndot/D: a cell whose absorption time is far below dt ends the
  step there (with D from its final ionisation state).
"""
import numpy as np

C = 2.99792458e10


def _case(O, smooth, sig):
    from paper_1304_7126_gb300 import workloads as W
    w = W.small_cosmo(10, seed=4, nsrc=2, flux=0)
    sigN = w.sigN if sig else np.zeros_like(w.sigN)
    sigE = w.sigE if sig else np.zeros_like(w.sigE)
    p = O.Problem(w.shape, w.dx, w.G, w.cr, sigN, sigE, w.egy, X=w.X, isothermal=w.isothermal,
                  otsa=True, flux=w.flux, bc=w.bc, smooth=smooth, nthreads=4)
    return w, p


def test_smooth_without_absorption_matches_unsmoothed(oracle_mod):
    O = oracle_mod
    w, ps = _case(O, True, False)
    _, pn = _case(O, False, False)
    dt = O.courant_dt(w.cfl, w.dx, w.cr)
    a, b = w.state(), w.state()
    for _ in range(3):
        assert ps.step(a, dt, w.src_ijk, w.src_L)[0] == 0
        assert pn.step(b, dt, w.src_ijk, w.src_L)[0] == 0
    scale = np.abs(b["N"]).max()
    assert np.max(np.abs(a["N"] - b["N"])) <= 1e-13 * scale
    assert np.max(np.abs(a["F"] - b["F"])) <= 1e-13 * w.cr * scale


def test_smooth_ledger(oracle_mod):
    O = oracle_mod
    w, p = _case(O, True, True)
    dt = O.courant_dt(w.cfl, w.dx, w.cr)
    s = w.state()
    prev = np.zeros(w.G)
    for _ in range(4):
        rc, b, sub, _ = p.step(s, dt, w.src_ijk, w.src_L)
        assert rc == 0
        # in_box(t + dt) = in_box(t) + emitted - absorbed - outflow
        np.testing.assert_allclose(b[:, 0], prev + b[:, 3] - b[:, 1] - b[:, 2], rtol=1e-12,
                                   atol=1e-12 * b[:, 3].max())
        prev = b[:, 0]
    assert b[:, 1].min() > 0.0


def test_smooth_fixed_point(oracle_mod):
    """One hydrogen-only cell, isothermal, a constant photon inflow rate:
    absorption and ionisation times (~1e9 s, ~1e12 s) << dt, so x settles
    and N ends at Ndot / D(x_final)."""
    O = oracle_mod
    sig = 1.63e-18
    cr = C / 100.0
    p = O.Problem((1, 1, 1), 1e21, 1, cr, [[sig, 0, 0]], [[1.1e-18, 0, 0]], [29.6 * 1.602176634e-12],
                  X=1.0, isothermal=True, otsa=True, flux=O.GLF, bc=(0,) * 6, smooth=True)
    nH, dt = 1.0, 1e15
    Ndot = 1e-13       # photons cm^-3 s^-1
    rc, s, N, F, att, ab, _ = p.thermo_cell(dt, nH, [1e-3, 0.0, 0.0, 1e4], [0.0], [[0.0, 0.0, 0.0]],
                                            Ndot=[Ndot], Fdot=[[0.0, 0.0, 0.0]])
    assert rc == 0
    D = cr * sig * nH * (1.0 - s[0])
    assert D * dt > 1e5
    # D of the last sub-step's start state, not of x_final: the last, long
    # sub-steps still move 1 - x by a few 1e-4
    np.testing.assert_allclose(N[0], Ndot / D, rtol=1e-3)
    # every photon that came in was either absorbed or is still there
    np.testing.assert_allclose(ab[0] + N[0], Ndot * dt, rtol=1e-10)

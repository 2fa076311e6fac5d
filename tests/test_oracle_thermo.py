"""Pins of the oracle's thermochemistry (Sec. 3.3 and App. A): closed-form
equilibria, the energy deposited per photo-ionisation, a hand-derived
sub-cycling schedule, and the photon ledger of a full step."""
import math

import numpy as np
import pytest

import analytic as A

C = 2.99792458e10
EV = 1.602176634e-12
K_B = 1.380649e-16


def _cell(O, G=1, sigN=((1.63e-18, 0, 0),), sigE=None, egy=(29.6 * EV,), X=1.0,
          isothermal=True, cr=C / 100.0, otsa=True):
    sigE = sigN if sigE is None else sigE
    return O.Problem((1, 1, 1), 1e20, G, cr, sigN, sigE, egy, X=X, isothermal=isothermal,
                     otsa=otsa)


def _converge(p, nH, s, N, F, dt, n=400, fixed=True):
    for _ in range(n):
        st, s, N, F, att, ab, mg = p.thermo_cell(dt, nH, s, N, F, fixed_photons=fixed)
        assert st == 0
    return s, N, F


@pytest.mark.parametrize("T", [1e4, 2e4, 5e4])
def test_collisional_ionisation_equilibrium(oracle_mod, T):
    """No photons, fixed T: x_HII -> beta/(alpha+beta) (Sec. 6 and the
    chemistry tests' CIE convergence)."""
    p = _cell(oracle_mod)
    r, _ = oracle_mod.rates(T)
    s, _, _ = _converge(p, 1.0, [1e-3, 0, 0, T], [0.0], np.zeros((1, 3)), 1e15)
    assert s[3] == T
    x_exact = r["beta_HI"] / (r["beta_HI"] + r["alpha_HII"])
    assert s[0] == pytest.approx(max(x_exact, 1e-6), rel=1e-10)


@pytest.mark.parametrize("N", [1e-7, 1e-6, 1e-4])
def test_photoionisation_equilibrium(oracle_mod, N):
    """Fixed photon density and temperature: x_HII is the root of
    n_H(alpha+beta)x^2 + (Gamma - beta n_H)x - Gamma = 0, Gamma = sigma c_r N."""
    T, nH, cr = 1e4, 1e-3, C / 100.0
    p = _cell(oracle_mod, cr=cr)
    r, _ = oracle_mod.rates(T)
    s, _, _ = _converge(p, nH, [1e-3, 0, 0, T], [N], np.zeros((1, 3)), 1e16)
    x_exact = A.photo_equilibrium_x(nH, r["alpha_HII"], r["beta_HI"], 1.63e-18 * cr * N)
    assert s[0] == pytest.approx(x_exact, rel=1e-10)


@pytest.mark.parametrize("T", [3e4, 6e4, 1.5e5])
def test_helium_equilibrium_ratios(oracle_mod, T):
    """Collisional (and photo-) equilibrium of helium at fixed T: the
    steady states of Eqs. (xheii_diff), (xheiii_diff) give
    x_HeII/x_HeI = (beta_HeI n_e + G_HeI)/(alpha_HeII n_e) and
    x_HeIII/x_HeII = (beta_HeII n_e + G_HeII)/(alpha_HeIII n_e)."""
    X, nH, cr = 0.76, 1e-2, C / 100.0
    sigN = ((1e-18, 2e-18, 5e-19),)
    for Nph in (0.0, 1e-6):
        p = _cell(oracle_mod, sigN=sigN, X=X, cr=cr)
        r, _ = oracle_mod.rates(T)
        s, _, _ = _converge(p, nH, [0.5, 0.3, 0.1, T], [Nph], np.zeros((1, 3)), 1e15, n=600)
        x, y2, y3 = s[0], s[1], s[2]
        y1 = 1.0 - y2 - y3
        nHe = nH * (1 - X) / (4 * X)
        ne = x * nH + (y2 + 2 * y3) * nHe
        G1 = sigN[0][1] * cr * Nph
        G2 = sigN[0][2] * cr * Nph
        assert y2 / y1 == pytest.approx((r["beta_HeI"] * ne + G1) / (r["alpha_HeII"] * ne), rel=1e-8)
        assert y3 / y2 == pytest.approx((r["beta_HeII"] * ne + G2) / (r["alpha_HeIII"] * ne), rel=1e-8)
        assert min(y1, y2, y3) >= 0.0 and y1 + y2 + y3 == pytest.approx(1.0, abs=1e-15)


def test_photoheating_energy_per_ionisation(oracle_mod):
    """Each photo-ionisation deposits (mean photon energy - 13.6 eV): over a
    short sub-step of cold neutral gas (negligible cooling),
    Delta(T/mu) = (gamma-1) Delta(eps) X / (n_H k_B), with
    Delta(eps) = n_HI sigma c_r N (egy - 13.6 eV) h (Eq. (PHeat2))."""
    egy = 20.0 * EV
    sig = 1.6e-18
    cr = C / 10.0
    p = _cell(oracle_mod, sigN=((sig, 0, 0),), egy=(egy,), isothermal=False, cr=cr)
    nH, N, T0, x0 = 1.0, 1e-9, 100.0, 1e-6
    h = 1e6
    st, s, _, _, att, _, _ = p.thermo_cell(h, nH, [x0, 0, 0, T0], [N], np.zeros((1, 3)),
                                           fixed_photons=True)
    assert st == 0 and att == 1
    mu0 = 1.0 / (1.0 + x0)
    mu1 = 1.0 / (1.0 + s[0])
    dTmu = s[3] / mu1 - T0 / mu0
    deps = nH * (1 - x0) * sig * cr * N * (egy - 13.6 * EV) * h
    expect = (2.0 / 3.0) * deps * 1.0 / (nH * K_B)
    assert dTmu == pytest.approx(expect, rel=1e-6)


def test_cooling_and_heating_signs(oracle_mod):
    """Ionised gas without radiation cools; cold neutral gas under a strong
    ionising field heats; isothermal mode never touches T."""
    p = _cell(oracle_mod, isothermal=False)
    st, s, _, _, _, _, _ = p.thermo_cell(1e12, 1.0, [1.0, 0, 0, 1e5], [0.0], np.zeros((1, 3)))
    assert st == 0 and s[3] < 1e5
    st, s, _, _, _, _, _ = p.thermo_cell(1e10, 1e-3, [1e-6, 0, 0, 100.0], [1e-2], np.zeros((1, 3)))
    assert st == 0 and s[3] > 100.0
    q = _cell(oracle_mod, isothermal=True)
    st, s, _, _, _, _, _ = q.thermo_cell(1e10, 1e-3, [1e-6, 0, 0, 1e4], [1e-2], np.zeros((1, 3)))
    assert s[3] == 1e4


def test_subcycle_schedule_pure_absorption(oracle_mod):
    """A cell whose only sizeable change is photo-absorption with
    D dt_RT = 1: the 10% rule halves dt four times (relative drops
    1/2, 1/3, 1/5, 1/9 all > 0.1), then 16 sub-steps of dt/16 pass with a
    drop 1/17 (> 5%, so no doubling): 20 attempts, N = N0 (16/17)^16, and the
    flux scales by the same factor (Eqs. (SIE photons))."""
    X, nH = 0.76, 1.0
    nHe = nH * (1 - X) / (4 * X)
    cr = C
    dt = 1e8
    sig = 1.0 / (dt * cr * nHe)          # D = c sigma n_HeII = 1/dt with x_HeII = 1
    p = _cell(oracle_mod, sigN=((0.0, 0.0, sig),), X=X, cr=cr)
    N0 = 1e-8
    F0 = np.array([[0.3 * cr * N0, 0.0, 0.0]])
    st, s, N, F, att, ab, mg = p.thermo_cell(dt, nH, [1.0, 1.0, 0.0, 1e4], [N0], F0)
    assert st == 0
    assert att == 20
    fac = (16.0 / 17.0) ** 16
    assert N[0] == pytest.approx(N0 * fac, rel=1e-4)
    assert F[0, 0] == pytest.approx(F0[0, 0] * N[0] / N0, rel=1e-12)
    # absorbed photons = photons removed
    assert ab[0] == pytest.approx(N0 - N[0], rel=1e-12)


def test_no_change_takes_one_attempt(oracle_mod):
    p = _cell(oracle_mod)
    r, _ = oracle_mod.rates(1e4)
    x = r["beta_HI"] / (r["beta_HI"] + r["alpha_HII"])
    st, s, N, F, att, _, _ = p.thermo_cell(1e12, 1e-3, [max(x, 1e-6), 0, 0, 1e4], [0.0],
                                           np.zeros((1, 3)))
    assert st == 0 and att == 1


def test_photon_ledger_full_step(oracle_mod):
    """Emitted = change in the box + absorbed + outflow, per group, over
    several full RT steps (H+He, evolving T, HLL, 3 groups)."""
    from paper_1304_7126_gb300 import workloads as W
    O = oracle_mod
    w = W.small_cosmo(10, seed=2, nsrc=3)
    p = O.Problem(w.shape, w.dx, w.G, w.cr, w.sigN, w.sigE, w.egy, X=w.X,
                  isothermal=w.isothermal, otsa=w.otsa, flux=w.flux, bc=w.bc)
    s = w.state()
    V = w.dx ** 3
    dt = O.courant_dt(0.8, w.dx, w.cr)
    in0 = s["N"].reshape(w.G, -1).sum(axis=1) * V
    tot = np.zeros((w.G, 4))
    for _ in range(6):
        st, b, sub, mg = p.step(s, dt, w.src_ijk, w.src_L)
        assert st == 0
        tot[:, 1:] += b[:, 1:]
        tot[:, 0] = b[:, 0]
    resid = tot[:, 3] - (tot[:, 0] - in0) - tot[:, 1] - tot[:, 2]
    assert np.all(np.abs(resid) <= 1e-12 * tot[:, 3])
    assert np.all(tot[:, 1] > 0) and sub.max() > 1

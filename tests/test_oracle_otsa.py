"""Pins of the oracle without the on-the-spot approximation (Sec. 3.3.2):
case A recombination rates and recombination photons C_i = sum_j b_ji
(alpha^A_j - alpha^B_j) n_j n_e (Eqs. (thchem_N), (cool_N_cr)).

* A closed one-cell box (periodic, no sources) at fixed T whose own
  recombination photons are absorbed in it reaches the case-B collisional
  equilibrium x = beta / (alpha^B + beta): every recombination straight to
  the ground state is undone by the photon it emits, which is what the
  on-the-spot approximation assumes.  If the photons cannot be absorbed
  (zero cross-section), the case-A equilibrium beta / (alpha^A + beta) is
  reached instead and the photons pile up in the box.
* The photon ledger closes with the recombination photons counted in the
  absorbed column (absorbed minus created).
"""
import numpy as np

C = 2.99792458e10
EV = 1.602176634e-12


def _cell(O, sig, otsa):
    return O.Problem((1, 1, 1), 1e24, 1, C / 10.0, [[sig, 0, 0]], [[0.9 * sig, 0, 0]], [13.6 * EV * 1.2],
                     X=1.0, isothermal=True, otsa=otsa, flux=O.GLF, bc=(2,) * 6)


def _run_cell(O, p, T, steps):
    """Returns the state and the photon budget summed over the steps."""
    s = O.new_state((1, 1, 1), 1, 1.0, 0.5, T)
    dt = O.courant_dt(0.8, 1e24, C / 10.0)
    tot = np.zeros((1, 4))
    for _ in range(steps):
        rc, b, sub, _ = p.step(s, dt)
        assert rc == 0
        tot[:, 1:] += b[:, 1:]
        tot[:, 0] = b[:, 0]
    return s, tot


def test_non_otsa_absorbed_recombination_photons_give_case_b_equilibrium(oracle_mod):
    O = oracle_mod
    T = 2.0e4
    s, _ = _run_cell(O, _cell(O, 1e-14, False), T, 20)
    r, _ = O.rates(T, case_b=True)
    xB = r["beta_HI"] / (r["alpha_HII"] + r["beta_HI"])
    np.testing.assert_allclose(s["xHII"][0], xB, rtol=1e-6)


def test_non_otsa_escaping_photons_give_case_a_equilibrium(oracle_mod):
    O = oracle_mod
    T = 2.0e4
    s, b = _run_cell(O, _cell(O, 0.0, False), T, 20)
    rA, _ = O.rates(T, case_b=False)
    rB, _ = O.rates(T, case_b=True)
    xA = rA["beta_HI"] / (rA["alpha_HII"] + rA["beta_HI"])
    xB = rB["beta_HI"] / (rB["alpha_HII"] + rB["beta_HI"])
    np.testing.assert_allclose(s["xHII"][0], xA, rtol=1e-6)
    assert abs(xA - xB) > 1e-2
    # nothing absorbs them: the photons created are all still there
    assert s["N"][0] > 0.0
    np.testing.assert_allclose(b[0, 0], -b[0, 1], rtol=1e-10)


def test_otsa_gives_case_b_equilibrium(oracle_mod):
    O = oracle_mod
    T = 2.0e4
    s, _ = _run_cell(O, _cell(O, 1e-14, True), T, 20)
    r, _ = O.rates(T, case_b=True)
    np.testing.assert_allclose(s["xHII"][0], r["beta_HI"] / (r["alpha_HII"] + r["beta_HI"]), rtol=1e-6)
    assert s["N"][0] == 0.0


def test_non_otsa_ledger(oracle_mod):
    from paper_1304_7126_gb300 import workloads as W
    O = oracle_mod
    w = W.small_cosmo(10, seed=4, nsrc=2, flux=0)
    p = O.Problem(w.shape, w.dx, w.G, w.cr, w.sigN, w.sigE, w.egy, X=w.X, isothermal=w.isothermal,
                  otsa=False, flux=w.flux, bc=w.bc, nthreads=4)
    dt = O.courant_dt(w.cfl, w.dx, w.cr)
    s = w.state()
    prev = np.zeros(w.G)
    for _ in range(4):
        rc, b, _, _ = p.step(s, dt, w.src_ijk, w.src_L)
        assert rc == 0
        np.testing.assert_allclose(b[:, 0], prev + b[:, 3] - b[:, 1] - b[:, 2], rtol=1e-12,
                                   atol=1e-12 * b[:, 3].max())
        prev = b[:, 0]

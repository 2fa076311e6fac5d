"""Pins of the oracle's inflow boundary (a face held at a given photon
state; the paper's fixed ionising flux entering the box, Sec. 6 test 3).

* A plane beam with f = 1 entering an empty box through the x = 0 face is
  exact upwinding at Courant number nu: N_i^n = N_in P(K >= i + 1),
  K ~ Binomial(n, nu) (the ghost cell i = -1 holds N_in), F = c N behind
  the front, for GLF and HLL; the photons that came in are the inflow
  tallied (negative outflow) at that face.
* Plane-parallel Stromgren length: a column of uniform hydrogen at fixed
  T under a constant flux F ionises until recombinations balance the
  incoming photons, sum alpha_B x^2 n_H^2 dx = F (to 1% after eight
  recombination times), i.e. to about l_S = F / (alpha_B n_H^2), 0.78 kpc
  for the paper's dense-cloud numbers (quoted in its test 3); the I-front
  (x_HII = 0.5) sits within 10% of l_S (it lies past l_S by the
  partial ionisation inside and the front's width).
"""
import numpy as np
import pytest
from scipy import stats

C = 2.99792458e10
EV = 1.602176634e-12
KPC = 3.0856775814913673e21


@pytest.mark.parametrize("flux", [0, 1])
def test_inflow_beam_is_exact_upwind(oracle_mod, flux):
    O = oracle_mod
    nx = 40
    shape = (2, 2, nx)
    cr = C / 100.0
    Nin = 3.0
    inflow = np.zeros((6, 1, 4))
    inflow[0, 0] = (Nin, cr * Nin, 0.0, 0.0)
    p = O.Problem(shape, 1e20, 1, cr, np.zeros((1, 3)), np.zeros((1, 3)), [3e-11], X=1.0, isothermal=True,
                  otsa=True, flux=flux, bc=(3, 0, 2, 2, 2, 2), skip_thermo=True, inflow=inflow)
    s = O.new_state(shape, 1, 1e-3, 1e-6, 1e4)
    dt = O.courant_dt(0.8, 1e20, cr)
    nu = cr * dt / 1e20
    n = 50
    inflow_total = 0.0
    for _ in range(n):
        _, b, _, _ = p.step(s, dt)
        inflow_total -= b[0, 2]
    N = s["N"].reshape(shape)
    F = s["F"].reshape((3,) + shape)
    exact = Nin * stats.binom.sf(np.arange(nx), n, nu)
    for z in range(2):
        for y in range(2):
            assert np.max(np.abs(N[z, y] - exact)) <= 1e-12 * Nin
            assert np.max(np.abs(F[0, z, y] - cr * N[z, y])) <= 1e-12 * cr * Nin
    # everything in the box came in through the x = 0 face
    np.testing.assert_allclose(inflow_total, N.sum() * 1e60, rtol=1e-12)


def test_plane_parallel_stromgren_length(oracle_mod):
    """One gray group (1.63e-18 cm^2), hydrogen only, T = 1e4 K fixed,
    n_H = 4e-2, F = 1e6 cm^-2 s^-1 through x = 0; 48 cells over 2 l_S;
    run 8 recombination times."""
    O = oracle_mod
    nH, Fin, T = 4e-2, 1e6, 1e4
    r, _ = O.rates(T, case_b=True)
    lS = Fin / (r["alpha_HII"] * nH * nH)
    assert lS / KPC == pytest.approx(0.78, rel=0.01)
    nx = 48
    dx = 2.0 * lS / nx
    cr = C / 10.0
    inflow = np.zeros((6, 1, 4))
    inflow[0, 0] = (Fin / cr, Fin, 0.0, 0.0)
    p = O.Problem((1, 1, nx), dx, 1, cr, [[1.63e-18, 0, 0]], [[1.1e-18, 0, 0]], [29.6 * EV], X=1.0,
                  isothermal=True, otsa=True, flux=O.HLL, bc=(3, 0, 2, 2, 2, 2), inflow=inflow)
    s = O.new_state((1, 1, nx), 1, nH, 1e-6, T)
    dt = O.courant_dt(0.8, dx, cr)
    t_rec = 1.0 / (r["alpha_HII"] * nH)
    steps = int(8 * t_rec / dt) + 1
    for _ in range(steps):
        assert p.step(s, dt)[0] == 0
    x = s["xHII"]
    recomb = float(np.sum(r["alpha_HII"] * (x * nH) ** 2) * dx)
    assert recomb / Fin == pytest.approx(1.0, abs=0.01)
    k = int(np.argmax(x < 0.5))
    assert 0 < k < nx
    front = (k - 1 + (x[k - 1] - 0.5) / (x[k - 1] - x[k]) + 0.5) * dx
    assert front / lS == pytest.approx(1.0, abs=0.1)

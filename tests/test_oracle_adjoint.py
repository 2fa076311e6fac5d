"""Pins of the oracle's finite-difference gradient (oracle/fd.py), the
reference the GPU adjoint is checked against.

* Transport alone (no absorption, periodic box): the photon count after K
  steps is sum_s L_s K dt exactly (injection Eq. (injnum); the telescoping
  flux sum of Eq. (dUdt_sol) leaves nothing through a closed box), so
  dJ/dL_s = K dt, and n_H does not enter at all.
* One isothermal cell without radiation, run for many recombination times:
  x_HII reaches collisional ionisation equilibrium x = beta/(alpha + beta),
  independent of n_H, so d M_HI / d n_H = m_H (1 - x) dx^3.
"""
import numpy as np
import pytest

C = 2.99792458e10


@pytest.fixture(scope="module")
def fd(oracle_mod):
    from oracle import fd as F
    return F


def test_fd_photon_count_transport_only(oracle_mod, fd):
    O = oracle_mod
    shape = (4, 5, 6)
    G = 2
    cr = C / 100.0
    p = O.Problem(shape, 1e20, G, cr, np.zeros((G, 3)), np.zeros((G, 3)), np.full(G, 3e-11), X=1.0,
                  isothermal=True, otsa=True, flux=O.GLF, bc=(2,) * 6, skip_thermo=True)
    s = O.new_state(shape, G, 1e-3, 1e-6, 1e4)
    rng = np.random.default_rng(4)
    s["N"][:] = 10 ** rng.uniform(-3, 0, size=s["N"].size)
    ijk = np.array([[1, 2, 3], [5, 0, 1]], dtype=np.int32)
    L = np.array([[2e48, 1e48], [5e47, 3e48]])
    dt = O.courant_dt(0.8, 1e20, cr)
    K = 4
    V = 1e60

    def count(st):
        return float(np.sum(st["N"]) * V)

    params = [("L", 0), ("L", 1), ("nH", 7)]
    g, info = fd.fd_gradient(p, s, dt, K, ijk, L, count, params)
    assert all(ok for _, ok in info)
    # J depends on L_s only through sum_i L_{s,i} K dt: dJ/dL_s = K dt
    np.testing.assert_allclose(g[:2], K * dt, rtol=1e-7)
    assert g[2] == 0.0


def test_fd_cie_cell_nH(oracle_mod, fd):
    O = oracle_mod
    T = 2.0e4
    dx = 1e24
    cr = C / 10.0
    p = O.Problem((1, 1, 1), dx, 1, cr, [[1.63e-18, 0, 0]], [[1.1e-18, 0, 0]], [29.6 * 1.602176634e-12],
                  X=1.0, isothermal=True, otsa=True, flux=O.GLF, bc=(0,) * 6)
    nH = 1.0
    s = O.new_state((1, 1, 1), 1, nH, 1e-3, T)
    dt = O.courant_dt(0.8, dx, cr)
    r, _ = O.rates(T)
    x_eq = r["beta_HI"] / (r["alpha_HII"] + r["beta_HI"])
    # many recombination times (1/(alpha n_e) ~ 1e12 s) at this dt
    K = 12
    assert K * dt * r["alpha_HII"] * nH * x_eq > 50.0
    g, info = fd.fd_gradient(p, s, dt, K, np.zeros((0, 3)), np.zeros((0, 1)),
                             lambda st: fd.neutral_hydrogen_mass(st, dx), [("nH", 0)])
    assert info[0][1]
    expect = fd.M_H * (1.0 - x_eq) * dx ** 3
    np.testing.assert_allclose(g[0], expect, rtol=1e-6)

"""Pins of the oracle's expansion-factor change (Problem.expand; Sec. 5,
cosmological settings: super-comoving photon variables N~ = a^3 N,
F~ = a^4 F / (H0 L), gas at constant comoving density).

* The super-comoving variables are unchanged by expand, and the photon
  count sum N V (V the physical cell volume) is conserved through any
  sequence of expansions and transport steps in a closed box without
  absorption (transport conserves it between expansions; the dilution
  a^-3 and the growth of V a^3 cancel).
* The Compton term follows T_gamma = 2.727 / a: a gas at that temperature
  neither heats nor cools by it.
"""
import numpy as np

C = 2.99792458e10


def test_expand_keeps_supercomoving_state_and_photon_count(oracle_mod):
    O = oracle_mod
    shape = (5, 6, 7)
    G = 2
    cr = C / 10.0
    a0 = 0.1
    dx_com = 1e21
    p = O.Problem(shape, a0 * dx_com, G, cr, np.zeros((G, 3)), np.zeros((G, 3)), np.full(G, 3e-11), X=1.0,
                  isothermal=True, otsa=True, flux=O.HLL, bc=(2,) * 6, a_exp=a0, skip_thermo=True)
    rng = np.random.default_rng(9)
    s = O.new_state(shape, G, 1e-3, 1e-6, 1e4)
    s["N"][:] = 10 ** rng.uniform(-3, 0, s["N"].size)
    d = rng.standard_normal((G, 3, s["N"].size // G))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    s["F"][:] = (cr * s["N"].reshape(G, 1, -1) * 0.5 * d).reshape(-1)
    count0 = s["N"].sum() * (a0 * dx_com) ** 3
    a = a0
    for a_new in (0.11, 0.125, 0.14):
        Nt, Ft = a ** 3 * s["N"].copy(), a ** 4 * s["F"].copy()
        p.expand(s, a_new)
        np.testing.assert_allclose(a_new ** 3 * s["N"], Nt, rtol=1e-14)
        np.testing.assert_allclose(a_new ** 4 * s["F"], Ft, rtol=1e-14, atol=1e-14 * np.abs(Ft).max())
        assert abs(p.cfg.dx / (a_new * dx_com) - 1.0) < 1e-14
        a = a_new
        dt = O.courant_dt(0.8, p.cfg.dx, cr)
        for _ in range(3):
            assert p.step(s, dt)[0] == 0
        np.testing.assert_allclose(s["N"].sum() * p.cfg.dx ** 3, count0, rtol=1e-12)


def test_compton_follows_the_expansion_factor(oracle_mod):
    O = oracle_mod
    for a in (1.0, 0.25, 0.1):
        Tg = 2.727 / a
        r, _ = O.rates(Tg, a_exp=a)
        assert abs(r["varpi"]) == 0.0
        r2, _ = O.rates(2.0 * Tg, a_exp=a)
        assert r2["varpi"] > 0.0

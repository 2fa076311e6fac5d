"""End-to-end pin of the oracle: the isothermal Stromgren sphere of the
paper's Sec. 6 test 1 (one octant, corner source, c_r = c/100, GLF) against
the analytic front r_S (1 - exp(-t/t_rec))^(1/3), Eq. (r_analyt), and the
c_r-aware front law of Sec. 4.2, Eq. (Stromgr_w_rel).  Run at 16^3 to keep
the CPU suite short (same box, same physics, 13936 steps to 500 Myr)."""
import json
import os

import pytest

import analytic as A

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_stromgren_front(oracle_mod):
    from paper_1304_7126_gb300 import workloads as W
    O = oracle_mod
    w = W.stromgren32(16)
    p = O.Problem(w.shape, w.dx, w.G, w.cr, w.sigN, w.sigE, w.egy, X=w.X,
                  isothermal=w.isothermal, otsa=w.otsa, flux=w.flux, bc=w.bc,
                  nthreads=min(8, os.cpu_count() or 1))
    s = w.state()
    dt = O.courant_dt(0.8, w.dx, w.cr)
    r, _ = O.rates(1e4)
    rS = A.stromgren_radius(w.extra["L_full"], 1e-3, r["alpha_HII"])
    tr = A.t_rec(1e-3, r["alpha_HII"])
    nsteps = int(round(w.extra["t_end_s"] / dt))
    checks = {int(round(t * A.MYR / dt)): t for t in (30.0, 100.0, 200.0)}
    checks[nsteps] = 500.0
    for k in range(1, nsteps + 1):
        st, _, _, _ = p.step(s, dt, w.src_ijk, w.src_L)
        assert st == 0
        if k in checks:
            t = k * dt
            rn = A.ifront_radius(s["xHII"].reshape(w.shape), w.dx)
            assert abs(rn / A.front_radius(t, rS, tr) - 1.0) <= 0.10, (checks[k], rn / rS)
            assert abs(rn / A.front_radius_relativistic(t, rS, tr, w.cr) - 1.0) <= 0.10
    # final radius: the paper's equilibrium front is 1.05 r_S
    assert 0.95 <= rn / rS <= 1.10
    assert s["T"].min() == 1e4 and s["T"].max() == 1e4

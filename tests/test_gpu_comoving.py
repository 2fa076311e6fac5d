"""rt_set_scale_factor (Sec. 5, cosmological settings: super-comoving
photon variables, gas at constant comoving density, T_gamma = 2.727/a in
the Compton term) on the GPU against the oracle's Problem.expand.

* A cosmological box (H+He, evolving T, sources) run from a = 0.1 with the
  expansion factor raised between steps: every field within 1e-10 of the
  oracle step by step, outside oracle-reported 10%/5% ties.
* A closed box without absorption: the photon count sum N V is conserved
  through expansions and steps (1e-12), as in the oracle.
"""
import numpy as np
import pytest

from parity import flux_err, oracle_problem, rel_err

pytestmark = pytest.mark.gpu
C = 2.99792458e10


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available()
    from paper_1304_7126_gb300 import rt
    rt.load()
    return rt


def test_expanding_box_parity(oracle_mod, R):
    from paper_1304_7126_gb300 import workloads as W
    w = W.small_cosmo(12, seed=8, nsrc=2, flux=1)
    a0 = 0.1
    sim = R.RT.from_workload(w, a_exp=a0)
    p = oracle_problem(oracle_mod, w, nthreads=4, a_exp=a0)
    ref = w.state()
    for step, a in enumerate((0.1, 0.102, 0.104, 0.107, 0.11)):
        sim.set_state(ref)
        if a != p.cfg.a_exp:
            sim.set_scale_factor(a)
            p.expand(ref, a)
        dt = sim.courant_dt()
        assert dt == pytest.approx(oracle_mod.courant_dt(w.cfl, p.cfg.dx, w.cr), rel=1e-14)
        sim.step(dt)
        st, b, sub_o, mg = p.step(ref, dt, w.src_ijk, w.src_L)
        assert st == 0
        tie = mg.reshape(-1) < 1e-12
        differ = (sim.subcycles() != sub_o).reshape(-1)
        assert np.all(tie[differ]), (step, int(differ.sum()))
        keep = ~tie
        kG = np.tile(keep, w.G)
        got = sim.get_state()
        for k in ("nH", "xHII", "xHeII", "T"):
            assert rel_err(got[k][keep], ref[k][keep]) < 1e-10, (step, k)
        assert rel_err(got["N"][kG], ref["N"][kG]) < 1e-10, step
        assert flux_err(got["F"].reshape(w.G, 3, -1)[:, :, keep], ref["F"].reshape(w.G, 3, -1)[:, :, keep],
                        ref["N"].reshape(w.G, -1)[:, keep], w.cr, w.G) < 1e-10, step
    # the reference state carries the expansion: a^3 N, nH comoving
    np.testing.assert_allclose(sim.get_state()["nH"] * 0.11 ** 3, w.nH * 0.1 ** 3, rtol=1e-13)


def test_expansion_conserves_photons(R):
    from paper_1304_7126_gb300 import workloads as W
    shape = (6, 6, 8)
    nc = int(np.prod(shape))
    G = 1
    w = W.Workload(name="closed", shape=shape, dx=1e20, G=G, cr=C / 10, sigN=np.zeros((G, 3)),
                   sigE=np.zeros((G, 3)), egy=np.full(G, 3e-11), X=1.0, isothermal=True, otsa=True, flux=0,
                   bc=(2,) * 6, steps=4)
    w.nH, w.xHII, w.T = np.full(nc, 1e-3), np.full(nc, 0.5), np.full(nc, 1e4)
    w.xHeII, w.xHeIII = np.zeros(nc), np.zeros(nc)
    w.src_ijk, w.src_L = np.zeros((0, 3), dtype=np.int32), np.zeros((0, G))
    sim = R.RT.from_workload(w, a_exp=0.5)
    rng = np.random.default_rng(3)
    s = w.state()
    s["N"] = 10 ** rng.uniform(-3, 0, nc)
    d = rng.standard_normal((3, nc))
    d /= np.linalg.norm(d, axis=0)
    s["F"] = (w.cr * s["N"] * 0.4 * d).reshape(-1)
    sim.set_state(s)
    count0 = s["N"].sum() * 1e60
    dx = 1e20
    for a in (0.55, 0.6, 0.7):
        sim.set_scale_factor(a)
        dx *= a / {0.55: 0.5, 0.6: 0.55, 0.7: 0.6}[a]
        for _ in range(3):
            sim.step(sim.courant_dt())
        np.testing.assert_allclose(sim.get_state()["N"].sum() * dx ** 3, count0, rtol=1e-12)

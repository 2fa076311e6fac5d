"""The inflow boundary (RT_BC_INFLOW: a face held at a given photon state,
the constant flux entering the box of the paper's Sec. 6 test 3) on the
GPU against the oracle.

* Transport only (all cross sections zero): a beam entering a box through
  x = 0 over a random photon field, GLF and HLL, within 1e-12 of the
  oracle, the inflow tallied as negative outflow; RT_MIXED within 1e-6.
* The dense-cloud workload (`workloads.shadow`) on a 16^3 grid, H only,
  evolving T, HLL: one step at a time from the oracle's state, 1e-10
  outside oracle-reported 10%/5% ties.
* The adjoint with an inflow face (the ghost is a given state, so it adds
  nothing to the cell's lambda): transport-only directional derivative
  against a central difference, GLF and HLL.
"""
import numpy as np
import pytest

from parity import compare, flux_err, oracle_problem, rel_err

pytestmark = pytest.mark.gpu
C = 2.99792458e10


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available()
    from paper_1304_7126_gb300 import rt
    rt.load()
    return rt


def _beam_case(shape, flux, G=2, seed=4):
    from paper_1304_7126_gb300 import workloads as W
    nz, ny, nx = shape
    nc = nx * ny * nz
    rng = np.random.default_rng(seed)
    w = W.Workload(name="beam", shape=shape, dx=3e20, G=G, cr=C / 100, sigN=np.zeros((G, 3)),
                   sigE=np.zeros((G, 3)), egy=np.full(G, 3e-11), X=1.0, isothermal=True, otsa=True, flux=flux,
                   bc=(3, 0, 2, 2, 1, 0), steps=4)
    w.nH = np.full(nc, 1e-3)
    w.xHII = np.full(nc, 0.5)
    w.xHeII = np.zeros(nc)
    w.xHeIII = np.zeros(nc)
    w.T = np.full(nc, 1e4)
    w.src_ijk = np.zeros((0, 3), dtype=np.int32)
    w.src_L = np.zeros((0, G))
    inflow = np.zeros((6, G, 4))
    inflow[0, :, 0] = [2.0, 0.5]
    inflow[0, :, 1] = w.cr * np.array([2.0, 0.5]) * 0.9
    inflow[0, :, 2] = w.cr * np.array([2.0, 0.5]) * 0.3
    w.extra = {"inflow": inflow}
    N = 10 ** rng.uniform(-3, 0, size=(G, nc))
    d = rng.standard_normal((G, 3, nc))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    F = w.cr * N[:, None, :] * rng.uniform(0.05, 0.9, size=(G, 1, nc)) * d
    return w, N.reshape(-1), F.reshape(-1)


@pytest.mark.parametrize("flux", [0, 1])
def test_inflow_transport_parity(oracle_mod, R, flux):
    w, N, F = _beam_case((7, 9, 12), flux)
    sim = R.RT.from_workload(w)
    s0 = w.state()
    s0["N"], s0["F"] = N.copy(), F.copy()
    sim.set_state(s0)
    mix = R.RT.from_workload(w, precision=R.RT_MIXED)
    mix.set_state(s0)
    p = oracle_problem(oracle_mod, w, skip_thermo=True)
    ref = {k: v.copy() for k, v in s0.items()}
    dt = sim.courant_dt()
    outflow = np.zeros(w.G)
    for _ in range(4):
        sim.step(dt)
        mix.step(dt)
        _, b, _, _ = p.step(ref, dt)
        outflow += b[:, 2]
        e = compare(sim.get_state(), ref, ("N", "F"), cr=w.cr, G=w.G)
        assert e["N"] < 1e-12 and e["F"] < 1e-12, e
    em = compare(mix.get_state(), ref, ("N", "F"), cr=w.cr, G=w.G)
    assert em["N"] < 1e-6 and em["F"] < 1e-6, em
    np.testing.assert_allclose(sim.budget()[:, 2], outflow, rtol=1e-10)
    assert outflow.min() < 0.0   # net inflow through x = 0


@pytest.mark.parametrize("otsa", [True, False])
def test_shadow_full_step_parity(oracle_mod, R, otsa):
    from paper_1304_7126_gb300 import workloads as W
    w = W.shadow(16, otsa=otsa)
    sim = R.RT.from_workload(w)
    p = oracle_problem(oracle_mod, w, nthreads=4)
    ref = w.state()
    dt = sim.courant_dt()
    for step in range(6):
        sim.set_state(ref)
        sim.step(dt)
        st, b, sub_o, mg = p.step(ref, dt, w.src_ijk, w.src_L)
        assert st == 0
        tie = mg.reshape(-1) < 1e-12
        differ = (sim.subcycles() != sub_o).reshape(-1)
        assert np.all(tie[differ]), (step, int(differ.sum()))
        keep = ~tie
        kG = np.tile(keep, w.G)
        got = sim.get_state()
        for k in ("xHII", "T"):
            assert rel_err(got[k][keep], ref[k][keep]) < 1e-10, (step, k)
        assert rel_err(got["N"][kG], ref["N"][kG]) < 1e-10, step
        assert flux_err(got["F"].reshape(w.G, 3, -1)[:, :, keep], ref["F"].reshape(w.G, 3, -1)[:, :, keep],
                        ref["N"].reshape(w.G, -1)[:, keep], w.cr, w.G) < 1e-10, step
    assert ref["N"].max() > 0.0


@pytest.mark.parametrize("flux", [0, 1])
def test_inflow_adjoint_directional(R, flux):
    import torch
    w, N, F = _beam_case((6, 7, 9), flux, seed=5)
    sim = R.RT.from_workload(w)
    s0 = w.state()
    s0["N"], s0["F"] = N.copy(), F.copy()
    dt = sim.courant_dt()
    nc, G = w.ncells, w.G
    rng = np.random.default_rng(6)
    vN = rng.standard_normal(G * nc)
    vF = rng.standard_normal(3 * G * nc) / w.cr
    uN = N * rng.standard_normal(G * nc)
    uF = w.cr * np.repeat(N.reshape(G, 1, nc), 3, axis=1).reshape(-1) * 0.05 * rng.standard_normal(3 * G * nc)

    def J(e):
        s = {k: v.copy() for k, v in s0.items()}
        s["N"] = N + e * uN
        s["F"] = F + e * uF
        sim.set_state(s)
        sim.step(dt)
        o = sim.get_state()
        return float(vN @ o["N"] + vF @ o["F"])

    eps = 1e-6 if flux == 0 else 1e-7
    fd = (J(eps) - J(-eps)) / (2 * eps)
    sim.set_state(s0)
    z = np.zeros(nc)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()  # noqa: E731
    lam = {"xHII": dev(z), "xHeII": dev(z), "xHeIII": dev(z), "T": dev(z), "N": dev(vN), "F": dev(vF)}
    sim.step_vjp(dt, lam, dev(z.copy()), None)
    torch.cuda.synchronize()
    ad = float(lam["N"].cpu().numpy() @ uN + lam["F"].cpu().numpy() @ uF)
    assert abs(ad - fd) <= (1e-6 if flux == 0 else 1e-5) * abs(fd), (ad, fd)

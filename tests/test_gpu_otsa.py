"""The RT step without the on-the-spot approximation (rt_options.otsa = 0,
Sec. 3.3.2): case-A rates and recombination photons C_i = sum_j b_ji
(alpha^A_j - alpha^B_j) n_j n_e (Eqs. (thchem_N), (cool_N_cr)).

* FP64 against the oracle, one step at a time from the oracle's state:
  every field within 1e-10 except in cells with an oracle-reported 10%/5%
  tie (none expected here), attempt counts equal elsewhere; GLF and HLL,
  H+He with evolving T and sources.
* A closed one-cell box whose recombination photons are absorbed in it
  reaches the case-B equilibrium beta/(alpha^B + beta) on the GPU as in
  the oracle (what the OTSA assumes).
* RT_MIXED and RT_MIXED32 within the stated tolerances of the FP64 path,
  and the photon ledger with the absorbed column net of created photons.
"""
import dataclasses

import numpy as np
import pytest

from parity import flux_err, oracle_problem, rel_err

pytestmark = pytest.mark.gpu
C = 2.99792458e10
EV = 1.602176634e-12


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available()
    from paper_1304_7126_gb300 import rt
    rt.load()
    return rt


def _cosmo(flux, seed=3):
    from paper_1304_7126_gb300 import workloads as W
    return dataclasses.replace(W.small_cosmo(16, seed=seed, nsrc=4, flux=flux, nx=21, ny=13), otsa=False)


@pytest.mark.parametrize("flux", [0, 1])
def test_non_otsa_parity_fp64(oracle_mod, R, flux):
    w = _cosmo(flux)
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
        for k in ("xHII", "xHeII", "xHeIII", "T"):
            assert rel_err(got[k][keep], ref[k][keep]) < 1e-10, (step, k)
        assert rel_err(got["N"][kG], ref["N"][kG]) < 1e-10, step
        assert flux_err(got["F"].reshape(w.G, 3, -1)[:, :, keep], ref["F"].reshape(w.G, 3, -1)[:, :, keep],
                        ref["N"].reshape(w.G, -1)[:, keep], w.cr, w.G) < 1e-10, step
        np.testing.assert_allclose(sim.budget()[:, 0], b[:, 0], rtol=1e-10)
    assert sub_o.max() > 1


def test_non_otsa_cell_reaches_case_b_equilibrium(oracle_mod, R):
    from paper_1304_7126_gb300 import workloads as W
    T = 2.0e4
    w = W.Workload(name="cell", shape=(1, 1, 1), dx=1e24, G=1, cr=C / 10.0, sigN=np.array([[1e-14, 0, 0]]),
                   sigE=np.array([[0.9e-14, 0, 0]]), egy=np.array([13.6 * EV * 1.2]), X=1.0, isothermal=True,
                   otsa=False, flux=0, bc=(2,) * 6, steps=20)
    w.nH, w.xHII, w.T = np.ones(1), np.full(1, 0.5), np.full(1, T)
    w.xHeII, w.xHeIII = np.zeros(1), np.zeros(1)
    w.src_ijk, w.src_L = np.zeros((0, 3), dtype=np.int32), np.zeros((0, 1))
    sim = R.RT.from_workload(w)
    dt = sim.courant_dt()
    for _ in range(20):
        sim.step(dt)
    x = sim.get_state()["xHII"][0]
    r, _ = oracle_mod.rates(T, case_b=True)
    np.testing.assert_allclose(x, r["beta_HI"] / (r["alpha_HII"] + r["beta_HI"]), rtol=1e-6)
    assert sim.get_state()["N"][0] > 0.0


@pytest.mark.parametrize("prec", ["mixed", "mixed32"])
def test_non_otsa_mixed_and_ledger(R, prec):
    from test_gpu_mixed import TOL
    w = _cosmo(1, seed=5)
    P = {"mixed": R.RT_MIXED, "mixed32": R.RT_MIXED32}[prec]
    ref_sim = R.RT.from_workload(w)
    sim = R.RT.from_workload(w, precision=P)
    dt = ref_sim.courant_dt()
    state = w.state()
    for _ in range(6):
        sim.set_state(state)
        ref_sim.set_state(state)
        sim.step(dt)
        ref_sim.step(dt)
        keep = (sim.subcycles() == ref_sim.subcycles()).reshape(-1)
        assert keep.mean() > 0.99
        got, ref = sim.get_state(), ref_sim.get_state()
        kG = np.tile(keep, w.G)
        for k in ("xHII", "xHeII", "xHeIII"):
            assert np.max(np.abs(got[k] - ref[k])[keep]) <= TOL[k], k
        assert rel_err(got["T"][keep], ref["T"][keep]) <= TOL["T"]
        assert rel_err(got["N"][kG], ref["N"][kG]) <= TOL["N"]
        state = ref
    # cumulative ledger of a run from the initial state
    s2 = R.RT.from_workload(w, precision=P)
    for _ in range(4):
        s2.step(dt)
    b = s2.budget()
    np.testing.assert_allclose(b[:, 0], b[:, 3] - b[:, 1] - b[:, 2], rtol=1e-6, atol=1e-6 * b[:, 3].max())

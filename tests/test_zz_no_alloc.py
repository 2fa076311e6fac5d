"""The allocation-free thermochemistry entry point against rt_step.

rt_thermo_step_noalloc serves callers that cannot allocate device memory
when they call in (for example code whose device memory is all reserved by
another framework's pool, or a loop that must keep a fixed footprint): it
runs the thermochemistry of one RT step on caller-owned device arrays with
its work queue in a fixed array inside the library.

Reference: for a photon field that is uniform in space with zero flux, the
transport of rt_step changes nothing (every face carries the same flux), so
rt_step on such a state is exactly its thermochemistry.  Two calls in a row
on different states must each match rt_step on the same state, within the
parity tolerance of the other GPU tests (1e-10 relative; identical
sub-cycle counts).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from parity import rel_err

pytestmark = pytest.mark.gpu


def _state(w, seed):
    """Uniform photons (F = 0), cell-to-cell varied gas."""
    rng = np.random.default_rng(seed)
    nc = w.ncells
    s = w.state()
    s["xHII"] = 10 ** rng.uniform(-6, 0, nc)
    y2 = rng.uniform(0, 0.6, nc)
    s["xHeII"] = y2
    s["xHeIII"] = rng.uniform(0, 1, nc) * (1 - y2) * 0.5
    s["T"] = 10 ** rng.uniform(2, 5.5, nc)
    s["N"] = np.repeat(10 ** rng.uniform(-9, -4, w.G), nc)
    s["F"] = np.zeros(3 * w.G * nc)
    return s


def test_noalloc_matches_rt_step_twice():
    import torch
    from paper_1304_7126_gb300 import rt as R
    from paper_1304_7126_gb300 import workloads as W

    w = W.small_cosmo(14, seed=9, nsrc=1, nx=29, ny=11)   # ragged 29 x 11 x 14
    opt = R.default_options(X=w.X, isothermal=0, otsa=1, flux=w.flux)
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((21, 22)):
        s = _state(w, seed)
        # existing entry point
        sim = R.RT.from_workload(w)
        sim.set_sources(None, None)
        sim.set_state(s)
        dt = sim.courant_dt()
        sim.step(dt)
        ref = sim.get_state()
        ref_sub = sim.subcycles().reshape(-1)
        sim.close()
        # allocation-free entry point on device copies of the same state
        dev = {k: torch.from_numpy(v.copy()).cuda() for k, v in s.items()}
        sub = torch.zeros(w.ncells, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        rc = R.rt_thermo_step_noalloc(w.ncells, w.G, opt, w.cr, w.sigN, w.sigE, w.egy, dt, dev, sub,
                                      stream.cuda_stream)
        assert rc == R.RT_OK, (call, rc)
        for k in ("N", "F", "xHII", "xHeII", "xHeIII", "T"):
            assert rel_err(dev[k].cpu().numpy(), ref[k]) <= 1e-10, (call, k)
        assert np.array_equal(sub.cpu().numpy(), ref_sub), call
        # cells past the first pass (6 attempts) and the first drain (128
        # more, the default routing) reach the second queue of the
        # library's array and, from there, the warp-per-cell kernel
        assert ref_sub.max() > 6 + 128, ("the state should make some cells sub-cycle long", int(ref_sub.max()))


def test_noalloc_rejects_too_many_cells():
    import torch
    from paper_1304_7126_gb300 import rt as R
    from paper_1304_7126_gb300 import workloads as W

    w = W.small_cosmo(8, seed=1, nsrc=1)
    opt = R.default_options(X=w.X)
    big = 262144 + 1
    dev = {k: torch.zeros(1, dtype=torch.float64, device="cuda")
           for k in ("nH", "xHII", "xHeII", "xHeIII", "T", "N", "F")}
    sub = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = R.rt_thermo_step_noalloc(big, w.G, opt, w.cr, w.sigN, w.sigE, w.egy, 1e10, dev, sub, None)
    assert rc == R.RT_EINVAL

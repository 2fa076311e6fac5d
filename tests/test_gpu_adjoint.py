"""The adjoint of the RT step (rt_step_vjp / rt_run_vjp through the C-ABI,
and the torch.autograd.Function on top) against finite differences.

* one step, transport only (all cross sections zero, so the photons pass
  the thermochemistry unchanged): <lambda_k, u> from the adjoint against
  the central difference of <v, U_{k+1}> along a random direction u, for
  outflow, reflecting and periodic boxes, GLF and HLL (whose wave speeds
  are differentiated through the bilinear table); and dJ/dL of the
  injection;
* one full step (H+He, evolving T, sources): the same directional check
  over every field and n_H, the sub-cycle schedule identical in the +/- runs
  and in the adjoint's recomputation; for HLL the photons of cells at a
  face with tied wave speeds (a kink of the step) are left unperturbed;
* several steps against the oracle's central-difference gradient of the
  neutral hydrogen mass (oracle/fd.py) with respect to n_H and the source
  luminosities;
* checkpointed autograd equals the unsegmented adjoint;
* the 64^3, 3-group, 8-source H+He workload over 10 steps: the autograd
  gradient of the neutral hydrogen mass against GPU central differences on
  random cells and all sources.
Gradient tolerance: 1e-4 relative (1e-6 for the smooth transport-only
case)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
C_LIGHT = 2.99792458e10
M_H = 1.67262192e-24


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available()
    from paper_1304_7126_gb300 import rt
    rt.load()
    return rt


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _transport_case(shape, bc, G, seed, flux=0):
    from paper_1304_7126_gb300 import workloads as W
    nz, ny, nx = shape
    nc = nx * ny * nz
    rng = np.random.default_rng(seed)
    w = W.Workload(name="tr", shape=shape, dx=3e20, G=G, cr=C_LIGHT / 100, sigN=np.zeros((G, 3)),
                   sigE=np.zeros((G, 3)), egy=np.full(G, 3e-11), X=1.0, isothermal=True, otsa=True,
                   flux=flux, bc=bc, steps=1)
    w.nH = np.full(nc, 1e-3)
    w.xHII = np.full(nc, 0.5)
    w.xHeII = np.zeros(nc)
    w.xHeIII = np.zeros(nc)
    w.T = np.full(nc, 1e4)
    N = 10 ** rng.uniform(-3, 0, size=(G, nc))
    d = rng.standard_normal((G, 3, nc))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    f = rng.uniform(0.05, 0.9, size=(G, 1, nc))
    F = w.cr * N[:, None, :] * f * d
    w.src_ijk = np.array([[1, 1, 1], [nx - 1, ny - 2, nz - 1]], dtype=np.int32)
    w.src_L = np.array([[3e50] * G, [1e50] * G])
    return w, N.reshape(-1), F.reshape(-1)


def _step_state(sim, s, dt):
    sim.set_state(s)
    sim.step(dt)
    return sim.get_state()


@pytest.mark.parametrize("flux", [0, 1])
@pytest.mark.parametrize("shape,bc", [((6, 7, 9), (0,) * 6), ((5, 6, 8), (1, 0, 2, 2, 0, 1)),
                                      ((8, 8, 8), (2,) * 6)])
def test_transport_vjp_directional(R, shape, bc, flux):
    import torch
    G = 2
    w, N, F = _transport_case(shape, bc, G, 21, flux)
    sim = R.RT.from_workload(w)
    s0 = w.state()
    s0["N"], s0["F"] = N.copy(), F.copy()
    dt = sim.courant_dt()
    nc = w.ncells
    rng = np.random.default_rng(22)
    vN = rng.standard_normal(G * nc)
    vF = rng.standard_normal(3 * G * nc) / w.cr
    uN = N * rng.standard_normal(G * nc)
    uF = (w.cr * np.repeat(N.reshape(G, 1, nc), 3, axis=1).reshape(-1)) * 0.05 * rng.standard_normal(3 * G * nc)

    def J(eps):
        s = {k: v.copy() for k, v in s0.items()}
        s["N"] = N + eps * uN
        s["F"] = F + eps * uF
        out = _step_state(sim, s, dt)
        return float(vN @ out["N"] + vF @ out["F"])

    # HLL: the speeds are piecewise (bilinear table cells, max / min), so a
    # shorter step keeps the difference inside one piece (rounding noise of
    # the difference ~1e-6 relative at this step)
    eps = 1e-6 if flux == 0 else 1e-7
    tol = 1e-6 if flux == 0 else 1e-5
    fd = (J(eps) - J(-eps)) / (2 * eps)
    sim.set_state(s0)
    lam = {"xHII": _dev(np.zeros(nc)), "xHeII": _dev(np.zeros(nc)), "xHeIII": _dev(np.zeros(nc)),
           "T": _dev(np.zeros(nc)), "N": _dev(vN), "F": _dev(vF)}
    g_nH = _dev(np.zeros(nc))
    g_L = _dev(np.zeros((2, G)))
    mism = sim.step_vjp(dt, lam, g_nH, g_L, check=True)
    torch.cuda.synchronize()
    ad = float(lam["N"].cpu().numpy() @ uN + lam["F"].cpu().numpy() @ uF)
    assert mism == 0
    assert abs(ad - fd) <= tol * abs(fd), (ad, fd)
    assert np.all(g_nH.cpu().numpy() == 0.0)
    # injection: dJ/dL_{s,i} = lambda_a(N_i at the source) dt / V; check by FD on L
    gL = g_L.cpu().numpy()
    for s_, i_ in ((0, 0), (1, 1)):
        def JL(eps):
            L = w.src_L.copy()
            L[s_, i_] *= 1 + eps
            sim.set_sources(w.src_ijk, L)
            v = J(0.0)
            sim.set_sources(w.src_ijk, w.src_L)
            return v
        fdl = (JL(1e-6) - JL(-1e-6)) / (2e-6 * w.src_L[s_, i_])
        assert abs(gL[s_, i_] - fdl) <= 1e-6 * abs(fdl), (s_, i_, gL[s_, i_], fdl)


def _evolved_cosmo(R, n, steps, seed=3, nsrc=2, flux=0):
    from paper_1304_7126_gb300 import workloads as W
    w = W.small_cosmo(n, seed=seed, nsrc=nsrc, flux=flux)
    sim = R.RT.from_workload(w)
    dt = sim.courant_dt()
    for _ in range(steps):
        sim.step(dt)
    return w, sim, dt, sim.get_state()


@pytest.mark.parametrize("flux", [0, 1])
def test_full_step_vjp_directional(R, oracle_mod, flux):
    import torch
    from parity import hll_tie_cells
    w, sim, dt, s0 = _evolved_cosmo(R, 10, 3, flux=flux)
    nc, G = w.ncells, w.G
    rng = np.random.default_rng(7)
    v = {"xHII": rng.standard_normal(nc), "xHeII": rng.standard_normal(nc), "xHeIII": rng.standard_normal(nc),
         "T": rng.standard_normal(nc) / 1e4, "N": rng.standard_normal(G * nc) / max(s0["N"].max(), 1e-300),
         "F": rng.standard_normal(3 * G * nc) / max(w.cr * s0["N"].max(), 1e-300)}
    # direction: relative perturbations of N, F, x_HII (kept inside [1e-6, 1], the
    # range rt_set_state accepts), T and n_H
    u = {"N": s0["N"] * rng.standard_normal(G * nc), "F": s0["F"] * rng.standard_normal(3 * G * nc) * 0.1,
         "xHII": np.minimum(s0["xHII"] - 1e-6, 1 - s0["xHII"]) * rng.standard_normal(nc),
         "T": s0["T"] * rng.standard_normal(nc), "nH": s0["nH"] * rng.standard_normal(nc)}
    if flux == 1:
        # HLL: at a face whose wave speeds tie (the photon front fills cells
        # with equal F/N) the step is only one-sidedly differentiable and a
        # central difference averages two slopes; move the photons of the
        # other cells only.  The tied cells exist (the front has reached
        # empty cells) but are few.
        tie = hll_tie_cells(oracle_mod, w, s0)
        assert 0 < tie.sum() < nc // 20
        for k in ("N", "F"):
            u[k] = u[k] * np.tile(~tie, u[k].size // nc)

    def J(eps):
        s = {k: a.copy() for k, a in s0.items()}
        for k, du in u.items():
            s[k] = s[k] + eps * du
        out = _step_state(sim, s, dt)
        return sum(float(v[k] @ out[k]) for k in v), sim.subcycles().copy()

    eps = 1e-7 if flux == 0 else 1e-8
    (jp, sp), (jm, sm) = J(eps), J(-eps)
    sim.set_state(s0)
    sim.step(dt)
    s_base = sim.subcycles().copy()
    assert np.array_equal(sp, sm) and np.array_equal(sp, s_base)
    fd = (jp - jm) / (2 * eps)
    sim.set_state(s0)
    lam = {k: _dev(v[k]) for k in ("xHII", "xHeII", "xHeIII", "T", "N", "F")}
    g_nH = _dev(np.zeros(nc))
    g_L = _dev(np.zeros((len(w.src_ijk), G)))
    mism = sim.step_vjp(dt, lam, g_nH, g_L, check=True)
    torch.cuda.synchronize()
    assert mism == 0
    ad = sum(float(lam[k].cpu().numpy() @ u[k]) for k in ("N", "F", "xHII", "T")) + \
        float(g_nH.cpu().numpy() @ u["nH"])
    assert s_base.max() > 6     # some cells sub-cycled
    assert abs(ad - fd) <= 1e-5 * abs(fd), (ad, fd)


def _gpu_mhi_grad(R, w, sim, dt, nsteps, s0):
    """dM_HI/dn_H (incl. the direct term) and dM_HI/dL[s][i] after nsteps."""
    import torch
    nc = w.ncells
    sim.set_state(s0)
    sim.run(dt, nsteps)
    fin = sim.get_state()
    V = w.dx ** 3
    lam = {"xHII": _dev(-M_H * s0["nH"] * V), "xHeII": _dev(np.zeros(nc)), "xHeIII": _dev(np.zeros(nc)),
           "T": _dev(np.zeros(nc)), "N": _dev(np.zeros(w.G * nc)), "F": _dev(np.zeros(3 * w.G * nc))}
    g_nH = _dev(M_H * (1.0 - fin["xHII"]) * V)
    g_L = _dev(np.zeros((len(w.src_ijk), w.G)))
    sim.set_state(s0)
    mism = sim.run_vjp(dt, nsteps, lam, g_nH, g_L, check=True)
    torch.cuda.synchronize()
    return g_nH.cpu().numpy(), g_L.cpu().numpy(), mism


@pytest.mark.parametrize("flux", [0, 1])
def test_run_vjp_against_oracle_fd(oracle_mod, R, flux):
    from oracle import fd as FD
    from parity import oracle_problem
    from paper_1304_7126_gb300 import workloads as W
    w = W.small_cosmo(8, seed=5, nsrc=2, flux=flux)
    sim = R.RT.from_workload(w)
    dt = sim.courant_dt()
    s0 = w.state()
    K = 4
    gN, gL, mism = _gpu_mhi_grad(R, w, sim, dt, K, s0)
    assert mism == 0
    p = oracle_problem(oracle_mod, w)
    rng = np.random.default_rng(5)
    src_cells = [int((k * w.shape[1] + j) * w.shape[2] + i) for i, j, k in w.src_ijk]
    cells = src_cells + [int(c) for c in rng.choice(w.ncells, 4, replace=False)]
    params = [("nH", c) for c in cells] + [("L", s) for s in range(len(w.src_ijk))]
    ref, info = FD.fd_gradient(p, s0, dt, K, w.src_ijk, w.src_L,
                               lambda st: FD.neutral_hydrogen_mass(st, w.dx), params)
    assert all(ok for _, ok in info)
    frac = w.src_L / w.src_L.sum(axis=1, keepdims=True)
    got = np.concatenate([gN[cells], (gL * frac).sum(axis=1)])
    nn = len(cells)
    for lo, hi in ((0, nn), (nn, len(params))):
        r, g = ref[lo:hi], got[lo:hi]
        scale = np.maximum(np.abs(r), 1e-3 * np.abs(r).max())
        assert np.all(np.abs(g - r) <= 1e-4 * scale), (params[lo:hi], g, r)


def test_autograd_checkpoints_match_unsegmented(R):
    import torch
    from paper_1304_7126_gb300 import adjoint as A
    from paper_1304_7126_gb300 import workloads as W
    w = W.small_cosmo(8, seed=6, nsrc=2, flux=0)
    sim = R.RT.from_workload(w)
    dt = sim.courant_dt()
    s0 = w.state()
    K = 6
    gN_ref, gL_ref, _ = _gpu_mhi_grad(R, w, sim, dt, K, s0)
    nH = _dev(s0["nH"]).requires_grad_(True)
    L = _dev(w.src_L).requires_grad_(True)
    st0 = {k: _dev(s0[k]) for k in A.STATE_KEYS}
    out = A.run(sim, dt, K, w.src_ijk, nH, L, st0, every=2)
    loss = A.neutral_hydrogen_mass(out, w.dx)
    loss.backward()
    torch.cuda.synchronize()
    np.testing.assert_allclose(nH.grad.cpu().numpy(), gN_ref, rtol=1e-12, atol=0)
    np.testing.assert_allclose(L.grad.cpu().numpy(), gL_ref, rtol=1e-12, atol=0)


def test_adjoint64_against_gpu_fd(R):
    """The 64^3, 3-group, 8-source workload over 10 steps."""
    import torch
    from paper_1304_7126_gb300 import adjoint as A
    from paper_1304_7126_gb300 import workloads as W
    w = W.adjoint64()
    sim = R.RT.from_workload(w)
    dt = sim.courant_dt()
    s0 = w.state()
    K = 10
    nH = _dev(s0["nH"]).requires_grad_(True)
    L = _dev(w.src_L).requires_grad_(True)
    st0 = {k: _dev(s0[k]) for k in A.STATE_KEYS}
    out = A.run(sim, dt, K, w.src_ijk, nH, L, st0, every=5)
    A.neutral_hydrogen_mass(out, w.dx).backward()
    torch.cuda.synchronize()
    gN, gL = nH.grad.cpu().numpy(), L.grad.cpu().numpy()
    frac = w.src_L / w.src_L.sum(axis=1, keepdims=True)
    gLs = (gL * frac).sum(axis=1)

    sub = torch.empty(w.ncells, dtype=torch.int32, device="cuda")

    def J(nHv, Lv):
        sim.set_sources(w.src_ijk, Lv)
        s = dict(s0)
        s["nH"] = nHv
        sim.set_state(s)
        scheds = []
        for _ in range(K):
            sim.step(dt)
            sim.L.rt_get_subcycles(sim.h, sub.data_ptr(), 1)
            scheds.append(sub.clone())
        fin = sim.get_state()
        # per-cell terms: the difference of the +/- runs is summed cell by
        # cell, so the unchanged cells cancel exactly
        return M_H * w.dx ** 3 * fin["nH"] * (1 - fin["xHII"]), torch.stack(scheds)

    def fd(mk, base):
        e = 1e-6 * base
        for _ in range(5):
            (jp, sp), (jm, sm) = J(*mk(e)), J(*mk(-e))
            if torch.equal(sp, sm):
                return float(np.sum(jp - jm)) / (2 * e)
            e *= 0.5
        raise AssertionError("no schedule-identical step")

    rng = np.random.default_rng(5)
    cells = [int(c) for c in rng.choice(w.ncells, 4, replace=False)]
    for c in cells:
        def mk(e, c=c):
            a = s0["nH"].copy()
            a[c] += e
            return a, w.src_L
        ref = fd(mk, s0["nH"][c])
        assert abs(gN[c] - ref) <= 1e-4 * abs(ref), (c, gN[c], ref)
    for s in range(len(w.src_ijk)):
        Ls = w.src_L[s].sum()

        def mk(e, s=s):
            Lv = w.src_L.copy()
            Lv[s] = w.src_L[s] * (Ls + e) / Ls
            return s0["nH"], Lv
        ref = fd(mk, Ls)
        assert abs(gLs[s] - ref) <= 1e-4 * abs(ref), (s, gLs[s], ref)

"""The adjoint workload as specified: 64^3, 3 groups, H+He, 8 sources, GLF,
200 FP64 steps, gradient of the neutral hydrogen mass
M_HI = sum m_H n_H (1 - x_HII) dx^3 at the end with respect to n_H at 32
cells drawn with default_rng(5) and to the luminosity of each of the 8
sources (at fixed spectral shape), through the torch.autograd front end
with a checkpoint every 20 steps, against central finite differences of the
GPU forward run with relative step 1e-6 for n_H (quartered until the two runs take the
same sub-cycle schedule in every cell and step; 1e-9 for a luminosity),
to 1e-4 relative.

The finite-difference runs are independent handles on their own streams,
advanced step by step together, so their serial thermochemistry tails
overlap on the GPU."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
M_H = 1.67262192e-24


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available()
    from paper_1304_7126_gb300 import rt
    rt.load()
    return rt


def _runs(R, w, K, inputs):
    """Advance one handle per (nH, L) input K steps together; the inputs come
    in (+, -) pairs.  Returns the per-cell M_HI terms at the end and, per
    pair, whether both runs took the same attempt count in every cell and
    step (the same sub-cycle schedule)."""
    sims = []
    for nHv, Lv in inputs:
        s = R.RT.from_workload(w)
        st = w.state()
        st["nH"] = nHv
        s.set_state(st)
        s.set_sources(w.src_ijk, Lv)
        sims.append(s)
    dt = sims[0].courant_dt()
    same = [True] * (len(sims) // 2)
    for _ in range(K):
        for s in sims:
            s.step(dt)
        for i in range(len(same)):
            a = sims[2 * i].subcycles()
            b = sims[2 * i + 1].subcycles()
            same[i] = same[i] and bool(np.array_equal(a, b))
    out = []
    for s in sims:
        fin = s.get_state()
        out.append(M_H * w.dx ** 3 * fin["nH"] * (1.0 - fin["xHII"]))
        s.close()
    return out, same


def test_adjoint64_200_steps_against_central_differences(R):
    import torch
    from paper_1304_7126_gb300 import adjoint as A
    from paper_1304_7126_gb300 import workloads as W
    w = W.adjoint64()
    K = 200
    sim = R.RT.from_workload(w)
    dt = sim.courant_dt()
    s0 = w.state()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    nH = dev(s0["nH"]).requires_grad_(True)
    L = dev(w.src_L).requires_grad_(True)
    out = A.run(sim, dt, K, w.src_ijk, nH, L, {k: dev(s0[k]) for k in A.STATE_KEYS}, every=20)
    A.neutral_hydrogen_mass(out, w.dx).backward()
    torch.cuda.synchronize()
    gN, gL = nH.grad.cpu().numpy(), L.grad.cpu().numpy()
    sim.close()
    frac = w.src_L / w.src_L.sum(axis=1, keepdims=True)
    gLs = (gL * frac).sum(axis=1)          # d M_HI / d (total luminosity of source s)

    # a photon can ionise at most one hydrogen atom: |dM_HI/dL| <= m_H K dt
    assert np.all(np.abs(gLs) <= M_H * K * dt * (1 + 1e-9)), gLs

    cells = [int(c) for c in np.random.default_rng(5).choice(w.ncells, 32, replace=False)]
    params = [("cell", c) for c in cells] + [("src", s) for s in range(len(w.src_ijk))]
    # relative steps: 1e-6 of n_H; 1e-9 of a luminosity, whose change
    # reaches every cell the source's photons reach, so that no 10%/5%
    # decision of the 200 steps in the whole box is tipped (the per-cell
    # rounding noise of the difference stays ~1e-5 of it down to 1e-11)
    base = {p: ((1e-6 * s0["nH"][p[1]]) if p[0] == "cell" else 1e-9 * w.src_L[p[1]].sum()) for p in params}
    ref = {}
    pending = list(params)
    for _ in range(4):
        inputs = []
        for p in pending:
            for sgn in (1.0, -1.0):
                e = sgn * base[p]
                a, Lv = s0["nH"].copy(), w.src_L.copy()
                if p[0] == "cell":
                    a[p[1]] += e
                else:
                    Ls = w.src_L[p[1]].sum()
                    Lv[p[1]] = w.src_L[p[1]] * (Ls + e) / Ls
                inputs.append((a, Lv))
        J, same = _runs(R, w, K, inputs)
        again = []
        for i, p in enumerate(pending):
            if same[i]:
                # per-cell terms summed cell by cell: unchanged cells cancel exactly
                ref[p] = float(np.sum(J[2 * i] - J[2 * i + 1])) / (2 * base[p])
            else:
                base[p] *= 0.25
                again.append(p)
        pending = again
        if not pending:
            break
    assert not pending, ("no schedule-identical step", pending)
    bad = []
    for p in params:
        got = gN[p[1]] if p[0] == "cell" else gLs[p[1]]
        if not abs(got - ref[p]) <= 1e-4 * abs(ref[p]):
            bad.append((p, got, ref[p]))
    assert not bad, bad

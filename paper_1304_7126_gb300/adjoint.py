"""torch.autograd front end of the rtgb adjoint (rt_run_vjp in include/rt.h).

:class:`RTRun` runs ``nsteps`` RT steps of an :class:`~.rt.RT` handle as one
differentiable function of the hydrogen density n_H, the source
luminosities L[s][i] and the initial state, and returns the final state.
Its backward pass is the library's hand-written adjoint: the forward pass
keeps a checkpoint of the state every ``every`` steps (device copies), and
the backward pass walks the segments from the last one, restoring each
checkpoint and calling ``rt_run_vjp`` over the segment, which recomputes
the segment's states and sweeps them back.  Memory: one state per
checkpoint plus one segment of states inside the library.

Argument marshalling only: every step and every adjoint step runs in the
CUDA library.
"""
from __future__ import annotations

import torch

from . import rt as R

STATE_KEYS = ("xHII", "xHeII", "xHeIII", "T", "N", "F")


class RTRun(torch.autograd.Function):
    """final (xHII, xHeII, xHeIII, T, N, F) = RTRun.apply(sim, dt, nsteps,
    every, src_ijk, nH, L, xHII0, xHeII0, xHeIII0, T0, N0, F0).

    sim: an rt.RT handle (precision RT_FP64, the OTSA and no smoothing for
    the backward pass; flux RT_GLF or RT_HLL); src_ijk: int array [n][3]; nH [cells], L [n][G] and the initial
    state: CUDA float64 tensors in the library layout."""

    @staticmethod
    def forward(ctx, sim, dt, nsteps, every, src_ijk, nH, L, x0, y20, y30, T0, N0, F0):
        every = max(1, int(every))
        # the library works on torch's stream, so tensors are ready in order
        sim.set_stream(torch.cuda.current_stream().cuda_stream)
        sim.set_sources(src_ijk, L.detach().cpu().numpy())
        st = {"nH": nH.detach().contiguous(), "xHII": x0.detach().contiguous(),
              "xHeII": y20.detach().contiguous(), "xHeIII": y30.detach().contiguous(),
              "T": T0.detach().contiguous(), "N": N0.detach().contiguous(), "F": F0.detach().contiguous()}
        sim.set_state(st)
        ckpts = []
        done = 0
        while done < nsteps:
            k = min(every, nsteps - done)
            ckpts.append((sim.get_state(device=True), k))
            sim.run(dt, k)
            done += k
        out = sim.get_state(device=True)
        sim.sync()
        ctx.sim, ctx.dt, ctx.ckpts = sim, dt, ckpts
        ctx.nsrc = int(L.shape[0])
        return tuple(out[k] for k in STATE_KEYS)

    @staticmethod
    def backward(ctx, *grads):
        sim = ctx.sim
        sim.set_stream(torch.cuda.current_stream().cuda_stream)
        ref = ctx.ckpts[0][0]
        lam = {}
        for k, g in zip(STATE_KEYS, grads):
            lam[k] = (g.detach().clone().contiguous() if g is not None else torch.zeros_like(ref[k]))
        g_nH = torch.zeros_like(ref["nH"])
        g_L = torch.zeros((ctx.nsrc, sim.G), dtype=torch.float64, device=g_nH.device)
        for state, k in reversed(ctx.ckpts):
            sim.set_state(state)
            sim.run_vjp(ctx.dt, k, lam, g_nH, g_L)
        return (None, None, None, None, None, g_nH, g_L, lam["xHII"], lam["xHeII"], lam["xHeIII"], lam["T"],
                lam["N"], lam["F"])


def run(sim, dt, nsteps, src_ijk, nH, L, state0: dict, every: int = 20):
    """Differentiable nsteps-step run: returns the final state as a dict of
    tensors (keys STATE_KEYS, plus the input nH)."""
    outs = RTRun.apply(sim, dt, nsteps, every, src_ijk, nH, L, state0["xHII"], state0["xHeII"],
                       state0["xHeIII"], state0["T"], state0["N"], state0["F"])
    d = dict(zip(STATE_KEYS, outs))
    d["nH"] = nH
    return d


M_H = 1.67262192e-24   # g, the proton mass


def neutral_hydrogen_mass(state: dict, dx: float):
    """M_HI = sum m_H n_H (1 - x_HII) dx^3, a differentiable torch scalar."""
    return M_H * dx ** 3 * torch.sum(state["nH"] * (1.0 - state["xHII"]))

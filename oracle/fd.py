"""Central finite-difference gradients of the oracle's RT run (test
infrastructure only, like the rest of ``oracle/``).

A gradient from the oracle is, by definition here, the central difference
(J(p + e) - J(p - e)) / (2 e) of a scalar J of the state after ``nsteps``
oracle steps (:meth:`oracle.Problem.step`, paper Sec. 3) with respect to one
scalar parameter p at a time: the hydrogen density n_H of one cell, or the
luminosity of one source (all its groups scaled together, so the group split
is fixed).  The thermochemistry's sub-cycle schedule (the 10% rule, App. A)
is piecewise constant in p; a difference taken across a change of schedule
measures a jump, not a derivative, so both runs must take the same schedule
in every cell and step, and the step e is halved until they do.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O

M_H = 1.67262192e-24   # g, the proton mass (the paper's m_H)


def run(prob: "O.Problem", state0: dict, dt: float, nsteps: int, src_ijk, src_L):
    """nsteps oracle steps from a copy of state0.  Returns (state, schedule):
    schedule is the (nsteps, cells) int32 array of per-cell attempts."""
    st = {k: np.array(v, dtype=np.float64, copy=True) for k, v in state0.items()}
    sched = np.zeros((nsteps, prob.ncells), dtype=np.int32)
    for k in range(nsteps):
        rc, _, sub, _ = prob.step(st, dt, src_ijk, src_L)
        if rc != 0:
            raise RuntimeError("oracle step failed with status %d" % rc)
        sched[k] = sub.reshape(-1)
    return st, sched


def neutral_hydrogen_mass(state: dict, dx: float) -> float:
    """M_HI = sum over cells of m_H n_H (1 - x_HII) dx^3 (grams)."""
    return float(M_H * np.sum(state["nH"] * (1.0 - state["xHII"])) * dx ** 3)


def fd_gradient(prob, state0, dt, nsteps, src_ijk, src_L, loss, params, rel_step=1e-6, max_halvings=6):
    """Central differences of loss(final_state) for each parameter in params:
    ("nH", cell) or ("L", source).  Returns (grad, info) with info[i] the
    relative step used and whether a schedule-identical pair was found."""
    src_ijk = np.asarray(src_ijk, dtype=np.int32).reshape(-1, 3)
    src_L = np.asarray(src_L, dtype=np.float64).reshape(src_ijk.shape[0], prob.G)
    grad = np.zeros(len(params))
    info = []
    for i, (kind, idx) in enumerate(params):
        base = state0["nH"][idx] if kind == "nH" else float(src_L[idx].sum())
        rs = rel_step
        ok = False
        for _ in range(max_halvings + 1):
            e = rs * base
            out = []
            for sgn in (1.0, -1.0):
                s0 = {k: np.array(v, copy=True) for k, v in state0.items()}
                Ls = src_L.copy()
                if kind == "nH":
                    s0["nH"][idx] = base + sgn * e
                else:
                    Ls[idx] = src_L[idx] * ((base + sgn * e) / base)
                st, sched = run(prob, s0, dt, nsteps, src_ijk, Ls)
                out.append((loss(st), sched))
            if np.array_equal(out[0][1], out[1][1]):
                ok = True
                break
            rs *= 0.5
        grad[i] = (out[0][0] - out[1][0]) / (2.0 * e)
        info.append((rs, ok))
    return grad, info

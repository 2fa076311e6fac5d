"""Write tests/golden/op_counts.json: the algorithmic FP64 work of the RT
step as the oracle states it, counted by the op-counting build of the oracle
(opcount.py), per unit the benchmark reports:

* thermochemistry: flops per attempt (one thermo_step of App. A, accepted or
  rejected, with the sub-cycling bookkeeping of Sec. 3.3.1), averaged over
  the attempts of the first two RT steps of the 128^3 benchmark workload;
* transport: flops per cell-group of one transport step (Sec. 3.2: closure,
  GLF or HLL face fluxes, update, realisability), on a 32^3 box with photons
  in every cell (random N, F with |F| < c_r N), for GLF and HLL.

Run: python -m oracle.make_counts   (single-threaded; about a minute)
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import opcount as OC  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1304_7126_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "op_counts.json")


def _problem(w, **kw):
    return O.Problem(w.shape, w.dx, w.G, w.cr, w.sigN, w.sigE, w.egy, X=w.X, isothermal=w.isothermal,
                     otsa=w.otsa, flux=w.flux, bc=w.bc, nthreads=1, **kw)


def thermo_counts(w, steps=2):
    """Per attempt: (all counts of the steps minus their transport) / attempts."""
    dt = O.courant_dt(w.cfl, w.dx, w.cr)
    p = _problem(w)
    pt = _problem(w, skip_thermo=True)
    s = w.state()
    tot = {k: 0 for k in OC.FIELDS + ("flop",)}
    attempts = 0
    for _ in range(steps):
        s_tr = {k: v.copy() for k, v in s.items()}
        with OC.counting():
            pt.step(s_tr, dt, w.src_ijk, w.src_L)
            c_tr = OC.counts()
        with OC.counting():
            st, _, sub, _ = p.step(s, dt, w.src_ijk, w.src_L)
            c = OC.counts()
        assert st == 0
        for k in tot:
            tot[k] += c[k] - c_tr[k]
        attempts += int(sub.sum())
    return {k: v / attempts for k, v in tot.items()}, attempts


def transport_counts(flux, n=32, G=3, seed=1):
    w = W.small_cosmo(n, seed=seed, nsrc=1, flux=flux)
    rng = np.random.default_rng(seed)
    nc = w.ncells
    N = 10 ** rng.uniform(-6, 0, size=(G, nc))
    d = rng.standard_normal((G, 3, nc))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    F = w.cr * N[:, None, :] * rng.uniform(0, 0.99, size=(G, 1, nc)) * d
    s = w.state()
    s["N"], s["F"] = N.reshape(-1).copy(), F.reshape(-1).copy()
    p = _problem(w, skip_thermo=True)
    dt = O.courant_dt(w.cfl, w.dx, w.cr)
    with OC.counting():
        st, _, _, _ = p.step(s, dt)
        c = OC.counts()
    assert st == 0
    return {k: v / (nc * G) for k, v in c.items()}


def main():
    w = W.cosmo128()
    th, att = thermo_counts(w)
    out = {
        "_about": "Algorithmic FP64 operation counts of the RT step as the oracle states it (op-counting build "
                  "of rt_oracle.c, oracle/opcount.cpp), written by oracle/make_counts.py. flop = add + mul + "
                  "div + sqrt; exp, log, pow calls counted apart. The oracle evaluates every rate fit and its "
                  "T-derivative at each temperature it needs.",
        "thermo_per_attempt": dict(th, sample="first 2 RT steps of the 128^3 benchmark workload (%d attempts)" % att),
        "transport_per_cell_group": {
            "glf": transport_counts(W.GLF),
            "hll": transport_counts(W.HLL),
            "sample": "one transport step of a 32^3 box, 3 groups, photons in every cell (random N, |F| < c_r N)"},
    }
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()

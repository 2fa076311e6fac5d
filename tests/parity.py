"""Helpers shared by the GPU parity tests: run the oracle and the CUDA
library on the same seeded inputs and compare field by field.  Flux
components are measured against their local scale c_r N (flux_err): a
component can vanish while |F| does not, so a per-component relative error
would be meaningless there."""
import numpy as np

FIELDS = ("N", "F", "xHII", "xHeII", "xHeIII", "T")


def rel_err(g, o):
    """max |g - o| / max(|o|, 1e-6 max|o|) (the parity metric)."""
    g = np.asarray(g, dtype=np.float64).reshape(-1)
    o = np.asarray(o, dtype=np.float64).reshape(-1)
    scale = np.max(np.abs(o)) if o.size else 0.0
    if scale == 0.0:
        return float(np.max(np.abs(g))) if g.size else 0.0
    return float(np.max(np.abs(g - o) / np.maximum(np.abs(o), 1e-6 * scale)))


def oracle_problem(O, w, **kw):
    if w.extra and w.extra.get("inflow") is not None and "inflow" not in kw:
        kw["inflow"] = w.extra["inflow"]
    return O.Problem(w.shape, w.dx, w.G, w.cr, w.sigN, w.sigE, w.egy, X=w.X,
                     isothermal=w.isothermal, otsa=w.otsa, flux=w.flux, bc=w.bc, **kw)


def flux_err(gF, oF, oN, cr, G):
    """Flux components measured against their natural local scale c_r N:
    max |dF| / max(c_r N, 1e-6 max(c_r N)) over cells, components, groups."""
    gF = np.asarray(gF).reshape(G, 3, -1)
    oF = np.asarray(oF).reshape(G, 3, -1)
    sc = cr * np.asarray(oN).reshape(G, 1, -1)
    m = sc.max()
    if m == 0.0:
        return float(np.max(np.abs(gF - oF)))
    return float(np.max(np.abs(gF - oF) / np.maximum(sc, 1e-6 * m)))


def compare(got, ref, fields=FIELDS, cr=None, G=None):
    out = {k: rel_err(got[k], ref[k]) for k in fields if not (k == "F" and cr is not None)}
    if "F" in fields and cr is not None:
        out["F"] = flux_err(got["F"], ref["F"], ref["N"], cr, G)
    return out

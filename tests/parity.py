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


def hll_tie_cells(O, w, s, atol=1e-6):
    """Cells on either side of an interior face where the HLL wave-speed
    choice max(0, lmax_L, lmax_R) or min(0, lmin_L, lmin_R) is (within atol,
    in units of c_r) a tie, for any group and direction.  The one-step map
    has a kink there (its one-sided derivatives differ): photons running
    into an empty region fill every cell with the same F/N, so neighbouring
    cells share (f, n) exactly and their speeds tie.  A tie between two
    cells at or below the closure floor (f := 0, speeds fixed at -+1/sqrt 3
    whatever the perturbation) is no kink, nor are boundary faces with
    zero-gradient ghosts, which tie with themselves and move together."""
    from oracle import hll_table
    tab = hll_table.table()
    nz, ny, nx = w.shape
    nc = nx * ny * nz
    N = s["N"].reshape(w.G, nc)
    F = s["F"].reshape(w.G, 3, nc)
    lo = np.zeros((w.G, 3, nc))
    hi = np.zeros((w.G, 3, nc))
    for g in range(w.G):
        for c in range(nc):
            _, f, n = O.eddington(w.cr, N[g, c], F[g, :, c])
            for d in range(3):
                lo[g, d, c], hi[g, d, c] = O.hll_lookup(tab, f, n[d])
    shape = (w.G, 3, nz, ny, nx)
    lo, hi = lo.reshape(shape), hi.reshape(shape)
    live = (N > 1e-30).reshape(w.G, nz, ny, nx)
    tie = np.zeros((nz, ny, nx), dtype=bool)

    def near_tie(a, b, sign):
        # the two largest of (0, a, b) (sign = +1) or smallest (sign = -1) within atol
        v = np.sort(np.stack([np.zeros_like(a), sign * a, sign * b]), axis=0)
        return v[2] - v[1] <= atol

    for d, ax in ((0, 4), (1, 3), (2, 2)):   # d = x, y, z face direction; array axis
        n_ax = shape[ax]
        sl_l = [slice(None)] * 5
        sl_r = [slice(None)] * 5
        sl_l[ax] = slice(0, n_ax - 1)
        sl_r[ax] = slice(1, n_ax)
        L_hi, R_hi = hi[:, d][tuple(sl_l[:1] + sl_l[2:])], hi[:, d][tuple(sl_r[:1] + sl_r[2:])]
        L_lo, R_lo = lo[:, d][tuple(sl_l[:1] + sl_l[2:])], lo[:, d][tuple(sl_r[:1] + sl_r[2:])]
        moves = live[tuple(sl_l[:1] + sl_l[2:])] | live[tuple(sl_r[:1] + sl_r[2:])]
        t = np.any((near_tie(L_hi, R_hi, 1.0) | near_tie(L_lo, R_lo, -1.0)) & moves, axis=0)
        m = np.zeros((nz, ny, nx), dtype=bool)
        sl = [slice(None)] * 3
        sl[ax - 2] = slice(0, n_ax - 1)
        m[tuple(sl)] |= t
        sl[ax - 2] = slice(1, n_ax)
        m[tuple(sl)] |= t
        tie |= m
    return tie.reshape(-1)

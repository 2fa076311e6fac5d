"""Thin ctypes binding of the rtgb C-ABI (include/rt.h).

Argument marshalling only: every step of the RT path runs in the CUDA
library ``librtgb.so``.  The functions keep the C names (``rt_create``,
``rt_step`` ...); :class:`RT` wraps a handle for convenience.  Arrays may be
numpy float64 arrays (host) or CUDA torch tensors (device pointers); there
is no CPU fallback: a missing library raises at import of the handle.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

RT_OK, RT_EINVAL, RT_EDT, RT_ESUBCYCLE, RT_EQUEUE, RT_ECUDA, RT_ENOMEM, RT_ENONFINITE = \
    0, -1, -2, -3, -4, -5, -6, -7
RT_BC_OUTFLOW, RT_BC_REFLECT, RT_BC_PERIODIC, RT_BC_INFLOW = 0, 1, 2, 3
RT_GLF, RT_HLL = 0, 1
RT_FP64, RT_MIXED, RT_MIXED32 = 0, 1, 2
RT_REC_BY_BAND = -2
RT_MAX_GROUPS = 8

ERROR_NAMES = {0: "RT_OK", -1: "RT_EINVAL", -2: "RT_EDT", -3: "RT_ESUBCYCLE", -4: "RT_EQUEUE",
               -5: "RT_ECUDA", -6: "RT_ENOMEM", -7: "RT_ENONFINITE"}


class rt_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx_cm", C.c_double),
                ("bc", C.c_int * 6)]


class rt_options(C.Structure):
    _fields_ = [("X", C.c_double), ("isothermal", C.c_int), ("otsa", C.c_int), ("flux", C.c_int),
                ("cfl", C.c_double), ("precision", C.c_int), ("a_exp", C.c_double),
                ("max_subcycles", C.c_int), ("smooth", C.c_int), ("rec_group", C.c_int * 3)]


class RTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERROR_NAMES.get(code, "?"), code, msg))
        self.code = code


_lib = None


def load(build: bool = True):
    """Load librtgb.so (building it with nvcc first if needed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("librtgb.so is not built (run __graft_entry__.build())")
    L = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.c_void_p, C.c_void_p
    L.rt_default_options.argtypes = [C.POINTER(rt_options)]
    L.rt_default_options.restype = None
    L.rt_create.argtypes = [C.POINTER(rt_grid), C.c_int, C.POINTER(rt_options), C.c_double, dp, dp, dp,
                            C.POINTER(vp)]
    L.rt_destroy.argtypes = [vp]
    L.rt_destroy.restype = None
    L.rt_set_stream.argtypes = [vp, vp]
    L.rt_set_state.argtypes = [vp, dp, dp, dp, dp, dp, dp, dp, C.c_int]
    L.rt_get_state.argtypes = [vp, dp, dp, dp, dp, dp, dp, dp, C.c_int]
    L.rt_set_sources.argtypes = [vp, C.c_int, ip, dp]
    L.rt_courant_dt.argtypes = [vp, C.POINTER(C.c_double)]
    L.rt_step.argtypes = [vp, C.c_double]
    L.rt_run.argtypes = [vp, C.c_double, C.c_int]
    L.rt_get_budget.argtypes = [vp, dp]
    L.rt_get_subcycles.argtypes = [vp, ip, C.c_int]
    L.rt_sync.argtypes = [vp]
    L.rt_last_error.argtypes = [vp]
    L.rt_last_error.restype = C.c_char_p
    L.rt_hll_table.argtypes = [C.c_int, C.c_int, dp]
    L.rt_version.argtypes = []
    L.rt_fmath_eval.argtypes = [C.c_int, C.c_longlong, dp, dp, vp]
    L.rt_set_inflow.argtypes = [vp, C.c_int, dp]
    L.rt_set_scale_factor.argtypes = [vp, C.c_double]
    L.rt_step_vjp.argtypes = [vp, C.c_double, dp, dp, dp, dp, dp, dp, dp, dp, C.POINTER(C.c_longlong)]
    L.rt_run_vjp.argtypes = [vp, C.c_double, C.c_int, dp, dp, dp, dp, dp, dp, dp, dp, C.POINTER(C.c_longlong)]
    L.rt_thermo_step_noalloc.argtypes = [C.c_longlong, C.c_int, C.POINTER(rt_options), C.c_double, dp, dp,
                                         dp, C.c_double, dp, dp, dp, dp, dp, dp, dp, ip, vp]
    L.rt_thermo_step_noalloc.restype = C.c_int
    L.rt_batch_create.argtypes = [C.c_int, C.POINTER(rt_grid), C.POINTER(C.c_int), C.POINTER(rt_options),
                                  C.c_double, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                  C.POINTER(vp)]
    L.rt_batch_destroy.argtypes = [vp]
    L.rt_batch_destroy.restype = None
    L.rt_batch_set_stream.argtypes = [vp, vp]
    L.rt_batch_set_box_state.argtypes = [vp, C.c_int, dp, dp, dp, dp, dp, dp, dp, C.c_int]
    L.rt_batch_get_box_state.argtypes = [vp, C.c_int, dp, dp, dp, dp, dp, dp, dp, C.c_int]
    L.rt_batch_set_box_sources.argtypes = [vp, C.c_int, C.c_int, ip, dp]
    L.rt_batch_courant_dt.argtypes = [vp, C.POINTER(C.c_double)]
    L.rt_batch_step.argtypes = [vp, C.c_double]
    L.rt_batch_run.argtypes = [vp, C.c_double, C.c_int]
    L.rt_batch_get_budget.argtypes = [vp, C.c_int, dp]
    L.rt_batch_sync.argtypes = [vp]
    L.rt_batch_last_error.argtypes = [vp]
    L.rt_batch_last_error.restype = C.c_char_p
    L.rt_batch_autotune.argtypes = [vp, C.c_int]
    L.rt_batch_box_tiling.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    for name in ("rt_batch_create", "rt_batch_set_stream", "rt_batch_set_box_state", "rt_batch_get_box_state",
                 "rt_batch_set_box_sources", "rt_batch_courant_dt", "rt_batch_step", "rt_batch_run",
                 "rt_batch_get_budget", "rt_batch_sync", "rt_batch_autotune", "rt_batch_box_tiling"):
        getattr(L, name).restype = C.c_int
    L.rt_set_profiling.argtypes = [vp, C.c_int]
    L.rt_get_profile.argtypes = [vp, dp, dp]
    L.rt_set_thermo_routing.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_longlong]
    L.rt_rate_functions.argtypes = [C.c_int, dp]
    for name in ("rt_create", "rt_set_stream", "rt_set_state", "rt_get_state", "rt_set_sources",
                 "rt_courant_dt", "rt_step", "rt_run", "rt_get_budget", "rt_get_subcycles", "rt_sync",
                 "rt_hll_table", "rt_version", "rt_set_profiling", "rt_get_profile", "rt_set_thermo_routing",
                 "rt_rate_functions"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _ptr(a):
    """Raw address of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a.data_ptr())


def _is_dev(a):
    return a is not None and not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def rt_hll_table(nf: int = 257, nmu: int = 257) -> np.ndarray:
    out = np.zeros((nf, nmu, 2))
    rc = load().rt_hll_table(nf, nmu, _ptr(out))
    if rc:
        raise RTError(rc, "rt_hll_table")
    return out


def rt_thermo_step_noalloc(ncells, G, opt, cr, sigN, sigE, egy, dt, state: dict, subcycles,
                           stream=None) -> int:
    """Allocation-free thermochemistry on caller-owned device arrays (torch
    CUDA tensors, updated in place); returns the C status code."""
    sn = np.ascontiguousarray(sigN, dtype=np.float64).reshape(G, 3)
    se = np.ascontiguousarray(sigE, dtype=np.float64).reshape(G, 3)
    eg = np.ascontiguousarray(egy, dtype=np.float64).reshape(G)
    keys = ("nH", "xHII", "xHeII", "xHeIII", "T", "N", "F")
    return load().rt_thermo_step_noalloc(int(ncells), int(G), C.byref(opt), float(cr), _ptr(sn), _ptr(se),
                                         _ptr(eg), float(dt), *[_ptr(state[k]) for k in keys],
                                         _ptr(subcycles), stream)


def rate_functions(case_b: bool = True) -> np.ndarray:
    """rt_rate_functions: the kernels' rate-function constants, [32][7] =
    (Cc, c0, c1, c2, c3, c4, c5) per slot (see include/rt.h)."""
    L = load()
    out = np.zeros((32, 7))
    rc = L.rt_rate_functions(int(bool(case_b)), out.ctypes.data_as(C.c_void_p))
    if rc != RT_OK:
        raise RuntimeError("rt_rate_functions: %d" % rc)
    return out


def default_options(**kw) -> rt_options:
    o = rt_options()
    load().rt_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "rec_group":
            v = (C.c_int * 3)(*[int(a) for a in v])
        setattr(o, k, v)
    return o


class RT:
    """One rtgb handle: a uniform grid, its photon groups and options."""

    def __init__(self, shape, dx, G, cr, sigN, sigE, egy, bc=(0,) * 6, **opts):
        L = load()
        nz, ny, nx = shape
        self.shape = (nz, ny, nx)
        self.G = int(G)
        g = rt_grid()
        g.nx, g.ny, g.nz = nx, ny, nz
        g.dx_cm = float(dx)
        for i in range(6):
            g.bc[i] = int(bc[i])
        o = default_options(**opts)
        sn = np.ascontiguousarray(sigN, dtype=np.float64).reshape(G, 3)
        se = np.ascontiguousarray(sigE, dtype=np.float64).reshape(G, 3)
        eg = np.ascontiguousarray(egy, dtype=np.float64).reshape(G)
        h = C.c_void_p()
        rc = L.rt_create(C.byref(g), self.G, C.byref(o), float(cr), _ptr(sn), _ptr(se), _ptr(eg), C.byref(h))
        if rc:
            raise RTError(rc, "rt_create")
        self.h = h
        self.L = L

    @property
    def ncells(self):
        nz, ny, nx = self.shape
        return nz * ny * nx

    def _check(self, rc, what):
        if rc:
            raise RTError(rc, "%s: %s" % (what, self.L.rt_last_error(self.h).decode()))

    def close(self):
        if getattr(self, "h", None):
            self.L.rt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr):
        self._check(self.L.rt_set_stream(self.h, stream_ptr), "rt_set_stream")

    def set_state(self, s: dict):
        keys = ("nH", "xHII", "xHeII", "xHeIII", "T", "N", "F")
        dev = _is_dev(s["N"])
        args = [_ptr(s[k]) for k in keys]
        self._check(self.L.rt_set_state(self.h, *args, int(dev)), "rt_set_state")

    def get_state(self, out: dict | None = None, device=False) -> dict:
        nc, G = self.ncells, self.G
        if out is None:
            if device:
                import torch
                mk = lambda n: torch.empty(n, dtype=torch.float64, device="cuda")  # noqa: E731
            else:
                mk = lambda n: np.empty(n)  # noqa: E731
            out = {"nH": mk(nc), "xHII": mk(nc), "xHeII": mk(nc), "xHeIII": mk(nc), "T": mk(nc),
                   "N": mk(G * nc), "F": mk(3 * G * nc)}
        keys = ("nH", "xHII", "xHeII", "xHeIII", "T", "N", "F")
        dev = any(_is_dev(out.get(k)) for k in keys)
        self._check(self.L.rt_get_state(self.h, *[_ptr(out.get(k)) for k in keys], int(dev)), "rt_get_state")
        return out

    def set_sources(self, ijk, L):
        if ijk is None or len(ijk) == 0:
            self._check(self.L.rt_set_sources(self.h, 0, None, None), "rt_set_sources")
            return
        a = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
        l = np.ascontiguousarray(L, dtype=np.float64).reshape(a.shape[0], self.G)
        self._check(self.L.rt_set_sources(self.h, a.shape[0], _ptr(a), _ptr(l)), "rt_set_sources")

    def set_inflow(self, face: int, state):
        """Ghost state [G][4] = (N, Fx, Fy, Fz) of an RT_BC_INFLOW face."""
        a = np.ascontiguousarray(state, dtype=np.float64).reshape(self.G, 4)
        self._check(self.L.rt_set_inflow(self.h, int(face), _ptr(a)), "rt_set_inflow")

    def set_scale_factor(self, a: float):
        """rt_set_scale_factor: change the expansion factor to a."""
        self._check(self.L.rt_set_scale_factor(self.h, float(a)), "rt_set_scale_factor")

    def courant_dt(self) -> float:
        d = C.c_double()
        self._check(self.L.rt_courant_dt(self.h, C.byref(d)), "rt_courant_dt")
        return d.value

    def step(self, dt: float = 0.0):
        self._check(self.L.rt_step(self.h, float(dt)), "rt_step")

    def run(self, dt: float, nsteps: int):
        self._check(self.L.rt_run(self.h, float(dt), int(nsteps)), "rt_run")

    def budget(self) -> np.ndarray:
        b = np.zeros((self.G, 4))
        self._check(self.L.rt_get_budget(self.h, _ptr(b)), "rt_get_budget")
        return b

    def subcycles(self) -> np.ndarray:
        s = np.zeros(self.ncells, dtype=np.int32)
        self._check(self.L.rt_get_subcycles(self.h, _ptr(s), 0), "rt_get_subcycles")
        return s.reshape(self.shape)

    def set_thermo_routing(self, pass1_attempts=0, drain_budget=0, drain2_budget=0, drain2_min_cells=-1):
        """rt_set_thermo_routing: which kernel runs which attempts of a cell
        (never the arithmetic); 0 / -1 restore the defaults."""
        self._check(self.L.rt_set_thermo_routing(self.h, int(pass1_attempts), int(drain_budget),
                                                 int(drain2_budget), int(drain2_min_cells)),
                    "rt_set_thermo_routing")

    PHASES = ("inject", "transport", "thermo_pass1", "thermo_drain", "reduce", "finalize")

    def set_profiling(self, on: bool):
        self._check(self.L.rt_set_profiling(self.h, int(bool(on))), "rt_set_profiling")

    def profile(self) -> dict:
        ms = np.zeros(6)
        n = np.zeros(6, dtype=np.int64)
        self._check(self.L.rt_get_profile(self.h, _ptr(ms), _ptr(n)), "rt_get_profile")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(self.PHASES)}

    def sync(self):
        self._check(self.L.rt_sync(self.h), "rt_sync")

    LAM_KEYS = ("xHII", "xHeII", "xHeIII", "T", "N", "F")

    def step_vjp(self, dt: float, lam: dict, g_nH, g_L=None, check: bool = False):
        """rt_step_vjp: lam (CUDA float64 tensors keyed as LAM_KEYS) goes in
        as dJ/dU_{k+1} and is overwritten with dJ/dU_k; g_nH and g_L
        accumulate.  Returns the schedule-mismatch count when `check`."""
        m = C.c_longlong(0)
        args = [_ptr(lam[k]) for k in self.LAM_KEYS]
        self._check(self.L.rt_step_vjp(self.h, float(dt), *args, _ptr(g_nH), _ptr(g_L),
                                       C.byref(m) if check else None), "rt_step_vjp")
        return m.value if check else None

    def run_vjp(self, dt: float, nsteps: int, lam: dict, g_nH, g_L=None, check: bool = False):
        """rt_run_vjp over nsteps steps from the current state."""
        m = C.c_longlong(0)
        args = [_ptr(lam[k]) for k in self.LAM_KEYS]
        self._check(self.L.rt_run_vjp(self.h, float(dt), int(nsteps), *args, _ptr(g_nH), _ptr(g_L),
                                      C.byref(m) if check else None), "rt_run_vjp")
        return m.value if check else None

    @classmethod
    def from_workload(cls, w, **opts):
        o = dict(X=w.X, isothermal=int(w.isothermal), otsa=int(w.otsa), flux=w.flux, cfl=w.cfl)
        o.update(opts)
        r = cls(w.shape, w.dx, w.G, w.cr, w.sigN, w.sigE, w.egy, bc=w.bc, **o)
        r.set_state(w.state())
        r.set_sources(w.src_ijk, w.src_L)
        inflow = w.extra.get("inflow") if w.extra else None
        if inflow is not None:
            for face in range(6):
                if w.bc[face] == RT_BC_INFLOW:
                    r.set_inflow(face, inflow[face])
        return r


class RTBatch:
    """A batch of independent boxes (rt_batch_* C-ABI): one entry per box in
    `boxes`, each a workloads.Workload sharing dx, c_r and options."""

    def __init__(self, boxes, **opts):
        L = load()
        self.L = L
        w0 = boxes[0]
        o = dict(X=w0.X, isothermal=int(w0.isothermal), otsa=int(w0.otsa), flux=w0.flux, cfl=w0.cfl)
        o.update(opts)
        opt = default_options(**o)
        n = len(boxes)
        grids = (rt_grid * n)()
        ng = (C.c_int * n)()
        self._keep = []
        sn, se, eg = (C.c_void_p * n)(), (C.c_void_p * n)(), (C.c_void_p * n)()
        for i, w in enumerate(boxes):
            nz, ny, nx = w.shape
            grids[i].nx, grids[i].ny, grids[i].nz = nx, ny, nz
            grids[i].dx_cm = float(w.dx)
            for k in range(6):
                grids[i].bc[k] = int(w.bc[k])
            ng[i] = w.G
            a = np.ascontiguousarray(w.sigN, dtype=np.float64).reshape(w.G, 3)
            b = np.ascontiguousarray(w.sigE, dtype=np.float64).reshape(w.G, 3)
            e = np.ascontiguousarray(w.egy, dtype=np.float64).reshape(w.G)
            self._keep += [a, b, e]
            sn[i], se[i], eg[i] = _ptr(a), _ptr(b), _ptr(e)
        h = C.c_void_p()
        rc = L.rt_batch_create(n, grids, ng, C.byref(opt), float(w0.cr), sn, se, eg, C.byref(h))
        if rc:
            raise RTError(rc, "rt_batch_create")
        self.h = h
        self.boxes = boxes

    def _check(self, rc, what):
        if rc:
            raise RTError(rc, "%s: %s" % (what, self.L.rt_batch_last_error(self.h).decode()))

    def close(self):
        if getattr(self, "h", None):
            self.L.rt_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr):
        self._check(self.L.rt_batch_set_stream(self.h, stream_ptr), "rt_batch_set_stream")

    def set_box_state(self, i, s):
        keys = ("nH", "xHII", "xHeII", "xHeIII", "T", "N", "F")
        dev = _is_dev(s["N"])
        self._check(self.L.rt_batch_set_box_state(self.h, i, *[_ptr(s[k]) for k in keys], int(dev)),
                    "rt_batch_set_box_state")

    def get_box_state(self, i):
        w = self.boxes[i]
        nc, G = w.ncells, w.G
        out = {"nH": np.empty(nc), "xHII": np.empty(nc), "xHeII": np.empty(nc), "xHeIII": np.empty(nc),
               "T": np.empty(nc), "N": np.empty(G * nc), "F": np.empty(3 * G * nc)}
        keys = ("nH", "xHII", "xHeII", "xHeIII", "T", "N", "F")
        self._check(self.L.rt_batch_get_box_state(self.h, i, *[_ptr(out[k]) for k in keys], 0),
                    "rt_batch_get_box_state")
        return out

    def set_box_sources(self, i, ijk, L):
        w = self.boxes[i]
        a = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
        l = np.ascontiguousarray(L, dtype=np.float64).reshape(a.shape[0], w.G)
        self._check(self.L.rt_batch_set_box_sources(self.h, i, a.shape[0], _ptr(a), _ptr(l)),
                    "rt_batch_set_box_sources")

    def courant_dt(self):
        d = C.c_double()
        self._check(self.L.rt_batch_courant_dt(self.h, C.byref(d)), "rt_batch_courant_dt")
        return d.value

    def step(self, dt=0.0):
        self._check(self.L.rt_batch_step(self.h, float(dt)), "rt_batch_step")

    def run(self, dt, nsteps):
        self._check(self.L.rt_batch_run(self.h, float(dt), int(nsteps)), "rt_batch_run")

    def budget(self, i):
        b = np.zeros((self.boxes[i].G, 4))
        self._check(self.L.rt_batch_get_budget(self.h, i, _ptr(b)), "rt_batch_get_budget")
        return b

    def sync(self):
        self._check(self.L.rt_batch_sync(self.h), "rt_batch_sync")

    def autotune(self, trials=2):
        self._check(self.L.rt_batch_autotune(self.h, int(trials)), "rt_batch_autotune")

    def tiling(self, i):
        a, b = C.c_int(), C.c_int()
        self._check(self.L.rt_batch_box_tiling(self.h, i, C.byref(a), C.byref(b)), "rt_batch_box_tiling")
        return a.value, b.value

    @classmethod
    def from_workloads(cls, boxes, **opts):
        r = cls(boxes, **opts)
        for i, w in enumerate(boxes):
            r.set_box_state(i, w.state())
            r.set_box_sources(i, w.src_ijk, w.src_L)
        return r

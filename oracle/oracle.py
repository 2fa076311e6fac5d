"""Python front end of the FP64 CPU oracle (test infrastructure only).

Builds ``rt_oracle.c`` with gcc into ``liboracle.so`` beside it and exposes
plain numpy-facing wrappers.  Only the test-suite, the package smoke check
and the CPU-baseline leg of ``bench.py`` may import this module; the CUDA
product path never does.

Every function follows the paper (Rosdahl et al. 2013):
  * :func:`step`        - one RT step, Sec. 3 (injection, transport,
                          thermochemistry in that order)
  * :func:`thermo_cell` - sub-cycled thermochemistry of one cell, App. A
  * :func:`rates`       - rate-coefficient fits, appendix on rate coefficients
  * :func:`chi`, :func:`eddington` - M1 closure, Sec. 2
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "rt_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

GLF, HLL = 0, 1
BC_OUTFLOW, BC_REFLECT, BC_PERIODIC, BC_INFLOW = 0, 1, 2, 3
MAXG = 8

RATE_NAMES = [
    "beta_HI", "beta_HeI", "beta_HeII",
    "alpha_HII", "alpha_HeII", "alpha_HeIII",
    "zeta_HI", "zeta_HeI", "zeta_HeII",
    "eta_HII", "eta_HeII", "eta_HeIII",
    "psi_HI", "psi_HeII",
    "theta", "varpi", "omega_HeII",
]

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over cells is its only parallelism).
    -ffp-contract=off: every operation is rounded on its own, as written, so
    the oracle gives the same bits on every host (x86 and Arm alike)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "rt_oracle.h")), os.path.getmtime(__file__)
    ):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
        )
        os.replace(tmp, LIB)
    return LIB


class OracleCfg(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double),
        ("bc", C.c_int * 6),
        ("G", C.c_int),
        ("cr", C.c_double),
        ("sigN", C.POINTER(C.c_double)),
        ("sigE", C.POINTER(C.c_double)),
        ("egy", C.POINTER(C.c_double)),
        ("X", C.c_double),
        ("isothermal", C.c_int),
        ("otsa", C.c_int),
        ("flux", C.c_int),
        ("a_exp", C.c_double),
        ("max_subcycles", C.c_int),
        ("hll_table", C.POINTER(C.c_double)),
        ("hll_nf", C.c_int), ("hll_nmu", C.c_int),
        ("nthreads", C.c_int),
        ("skip_thermo", C.c_int),
        ("smooth", C.c_int),
        ("rec_group", C.c_int * 3),
        ("inflow", C.POINTER(C.c_double)),
    ]


def bind(L):
    """Declare the oracle's C signatures on a loaded library (the oracle, or
    its op-counting build, which exports the same functions)."""
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int32)
    L.oracle_rates.argtypes = [C.c_double, C.c_double, C.c_int, dp, dp]
    L.oracle_chi.argtypes = [C.c_double]
    L.oracle_chi.restype = C.c_double
    L.oracle_eddington.argtypes = [C.c_double, C.c_double, dp, dp, dp, dp]
    L.oracle_hll_lookup.argtypes = [dp, C.c_int, C.c_int, C.c_double, C.c_double, dp, dp]
    L.oracle_thermo_cell.argtypes = [C.POINTER(OracleCfg), C.c_double, C.c_double,
                                     dp, dp, dp, dp, dp, C.c_int, C.POINTER(C.c_int), dp, dp]
    L.oracle_courant_dt.argtypes = [C.c_double, C.c_double, C.c_double]
    L.oracle_courant_dt.restype = C.c_double
    L.oracle_step.argtypes = [C.POINTER(OracleCfg), C.c_double, dp, dp, dp, dp, dp, dp, dp,
                              C.c_int, ip, dp, dp, ip, dp]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = bind(C.CDLL(LIB))
        return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def rates(T: float, a_exp: float = 1.0, case_b: bool = True):
    """Rate fits and their T-derivatives at temperature T [K] -> (dict, dict)."""
    r = np.zeros(len(RATE_NAMES))
    dr = np.zeros(len(RATE_NAMES))
    lib().oracle_rates(float(T), float(a_exp), int(bool(case_b)), _dp(r), _dp(dr))
    return dict(zip(RATE_NAMES, r)), dict(zip(RATE_NAMES, dr))


def chi(f: float) -> float:
    """Eddington factor of the M1 closure, Eq. (Udir)."""
    return lib().oracle_chi(float(f))


def eddington(c: float, N: float, F) -> tuple[np.ndarray, float, np.ndarray]:
    """Eddington tensor D (3x3), reduced flux f and unit direction n."""
    Fa = np.ascontiguousarray(F, dtype=np.float64)
    D = np.zeros(9)
    f = np.zeros(1)
    n = np.zeros(3)
    lib().oracle_eddington(float(c), float(N), _dp(Fa), _dp(D), _dp(f), _dp(n))
    return D.reshape(3, 3), float(f[0]), n


def hll_lookup(table: np.ndarray, f: float, mu: float) -> tuple[float, float]:
    t = np.ascontiguousarray(table, dtype=np.float64)
    lo = np.zeros(1)
    hi = np.zeros(1)
    lib().oracle_hll_lookup(_dp(t), t.shape[0], t.shape[1], float(f), float(mu), _dp(lo), _dp(hi))
    return float(lo[0]), float(hi[0])


def courant_dt(cfl: float, dx: float, cr: float) -> float:
    return lib().oracle_courant_dt(float(cfl), float(dx), float(cr))


class Problem:
    """Grid + options + group constants of one oracle run.

    Arrays follow the library layout: scalars [nz][ny][nx] (x fastest),
    N [G][nz][ny][nx], F [G][3][nz][ny][nx].
    """

    def __init__(self, shape, dx, G, cr, sigN, sigE, egy, X=1.0, isothermal=False,
                 otsa=True, flux=GLF, bc=(0, 0, 0, 0, 0, 0), a_exp=1.0,
                 max_subcycles=1_000_000, hll_table=None, nthreads=1, skip_thermo=False, smooth=False,
                 rec_group=None, inflow=None):
        nz, ny, nx = shape
        self.shape = (nz, ny, nx)
        self.G = int(G)
        self._sigN = np.ascontiguousarray(np.asarray(sigN, dtype=np.float64).reshape(G, 3))
        self._sigE = np.ascontiguousarray(np.asarray(sigE, dtype=np.float64).reshape(G, 3))
        self._egy = np.ascontiguousarray(np.asarray(egy, dtype=np.float64).reshape(G))
        if flux == HLL and hll_table is None:
            from . import hll_table as _ht
            hll_table = _ht.table()
        self._tab = (np.ascontiguousarray(hll_table, dtype=np.float64)
                     if hll_table is not None else np.zeros((2, 2, 2)))
        cfg = OracleCfg()
        cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
        cfg.dx = float(dx)
        for i in range(6):
            cfg.bc[i] = int(bc[i])
        cfg.G = self.G
        cfg.cr = float(cr)
        cfg.sigN = _dp(self._sigN)
        cfg.sigE = _dp(self._sigE)
        cfg.egy = _dp(self._egy)
        cfg.X = float(X)
        cfg.isothermal = int(bool(isothermal))
        cfg.otsa = int(bool(otsa))
        cfg.flux = int(flux)
        cfg.a_exp = float(a_exp)
        cfg.max_subcycles = int(max_subcycles)
        cfg.hll_table = _dp(self._tab)
        cfg.hll_nf, cfg.hll_nmu = self._tab.shape[0], self._tab.shape[1]
        cfg.nthreads = int(nthreads)
        cfg.skip_thermo = int(bool(skip_thermo))
        cfg.smooth = int(bool(smooth))
        # without the OTSA: the group that HII, HeII, HeIII recombinations
        # emit into; by default the groups are taken as ordered by band, so
        # species j emits into group min(j, G - 1)
        rg = rec_group if rec_group is not None else [min(j, self.G - 1) for j in range(3)]
        for j in range(3):
            cfg.rec_group[j] = int(rg[j])
        # faces with bc = BC_INFLOW hold the ghost state inflow[face][group]
        # = (N, Fx, Fy, Fz)
        self._inflow = (np.ascontiguousarray(inflow, dtype=np.float64).reshape(6, G, 4)
                        if inflow is not None else None)
        cfg.inflow = _dp(self._inflow) if self._inflow is not None else None
        self.cfg = cfg

    @property
    def ncells(self):
        nz, ny, nx = self.shape
        return nz * ny * nx

    def step(self, state: dict, dt: float, src_ijk=None, src_L=None):
        """Advance ``state`` (dict of float64 arrays, modified in place) by one
        RT step.  Returns (status, budget[G][4], subcycles, margins).

        budget columns: photons in the box after the step, absorbed in the
        step, outflow through the box faces in the step, emitted in the step.
        """
        G = self.G
        nc = self.ncells
        for k in ("nH", "xHII", "xHeII", "xHeIII", "T"):
            assert state[k].dtype == np.float64 and state[k].flags.c_contiguous and state[k].size == nc
        assert state["N"].size == G * nc and state["F"].size == 3 * G * nc
        if src_ijk is None or len(src_ijk) == 0:
            ijk = np.zeros((1, 3), dtype=np.int32)
            L = np.zeros((1, G))
            ns = 0
        else:
            ijk = np.ascontiguousarray(src_ijk, dtype=np.int32).reshape(-1, 3)
            L = np.ascontiguousarray(src_L, dtype=np.float64).reshape(-1, G)
            ns = ijk.shape[0]
        budget = np.zeros((G, 4))
        sub = np.zeros(nc, dtype=np.int32)
        mg = np.zeros(nc)
        st = lib().oracle_step(
            C.byref(self.cfg), float(dt), _dp(state["nH"]), _dp(state["xHII"]),
            _dp(state["xHeII"]), _dp(state["xHeIII"]), _dp(state["T"]),
            _dp(state["N"]), _dp(state["F"]), ns,
            ijk.ctypes.data_as(C.POINTER(C.c_int32)), _dp(L), _dp(budget),
            sub.ctypes.data_as(C.POINTER(C.c_int32)), _dp(mg))
        return st, budget, sub.reshape(self.shape), mg.reshape(self.shape)

    def expand(self, state: dict, a_new: float):
        """Change the expansion factor to a_new (Sec. 5, cosmological
        settings).  The photon state is kept in the super-comoving
        variables N~ = a^3 N, F~ = a^4 F / (H0 L) and the gas at constant
        comoving density, so in physical units N scales by (a/a_new)^3, F by
        (a/a_new)^4 and n_H by (a/a_new)^3; the physical cell width becomes
        a_new times the comoving one, and the Compton term takes
        T_gamma = 2.727 / a_new.  With a fixed between two changes, the
        transport equations in those variables are the physical ones at
        that cell width, so the steps themselves are unchanged.  (The
        adiabatic cooling of the gas belongs to the hydrodynamics and is
        not applied.)  state is modified in place."""
        a_old = float(self.cfg.a_exp)
        r = a_old / float(a_new)
        state["N"] *= r ** 3
        state["F"] *= r ** 4
        state["nH"] *= r ** 3
        self.cfg.dx = float(self.cfg.dx) / r
        self.cfg.a_exp = float(a_new)

    def thermo_cell(self, dt: float, nH: float, s, N, F, fixed_photons=False, Ndot=None, Fdot=None):
        """Sub-cycle one cell over dt.  s = [x_HII, x_HeII, x_HeIII, T];
        N [G]; F [G][3]; Ndot [G], Fdot [G][3]: smoothed-RT rates (Sec. 3.4)
        or None.  Returns (status, s, N, F, attempts, absorbed, margin);
        absorbed is net of the recombination photons created without the
        OTSA."""
        s = np.array(s, dtype=np.float64)
        N = np.array(N, dtype=np.float64).reshape(self.G)
        F = np.array(F, dtype=np.float64).reshape(self.G, 3).copy()
        att = C.c_int(0)
        ab = np.zeros(self.G)
        mg = np.zeros(1)
        nd = None if Ndot is None else np.ascontiguousarray(Ndot, dtype=np.float64).reshape(self.G)
        fd = None if Fdot is None else np.ascontiguousarray(Fdot, dtype=np.float64).reshape(self.G, 3)
        st = lib().oracle_thermo_cell(C.byref(self.cfg), float(dt), float(nH), _dp(s), _dp(N),
                                      _dp(F), None if nd is None else _dp(nd), None if fd is None else _dp(fd),
                                      int(bool(fixed_photons)), C.byref(att), _dp(ab), _dp(mg))
        return st, s, N, F, att.value, ab, float(mg[0])


def new_state(shape, G, nH, xHII, T, xHeII=0.0, xHeIII=0.0):
    """Dense float64 state dict in the library layout."""
    nz, ny, nx = shape
    nc = nz * ny * nx

    def fill(v):
        a = np.empty(nc)
        a[:] = np.asarray(v, dtype=np.float64).reshape(-1) if np.ndim(v) else v
        return a

    return {
        "nH": fill(nH), "xHII": fill(xHII), "xHeII": fill(xHeII), "xHeIII": fill(xHeIII),
        "T": fill(T), "N": np.zeros(G * nc), "F": np.zeros(3 * G * nc),
    }

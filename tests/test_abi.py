"""The C-ABI library loads, exports every function include/rt.h declares,
and its host-side pieces (defaults, argument checks, HLL table) work
without a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rt_[a-z_0-9]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1304_7126_gb300 import rt as R
    return R.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert {"rt_create", "rt_step", "rt_get_state", "rt_set_sources", "rt_destroy"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_default_options(lib):
    from paper_1304_7126_gb300 import rt as R
    o = R.default_options()
    assert o.X == 0.76 and o.otsa == 1 and o.flux == R.RT_GLF and o.cfl == 0.8
    assert o.max_subcycles == 1000000 and o.precision == R.RT_FP64


def test_create_rejects_bad_arguments(lib):
    from paper_1304_7126_gb300 import rt as R
    g = R.rt_grid()
    g.nx, g.ny, g.nz, g.dx_cm = 0, 4, 4, 1.0
    o = R.default_options()
    z = np.zeros(3)
    h = C.c_void_p()
    # checked on the host before any CUDA call
    assert lib.rt_create(C.byref(g), 1, C.byref(o), 1e9, z.ctypes.data, z.ctypes.data,
                         np.ones(1).ctypes.data, C.byref(h)) == R.RT_EINVAL
    g.nx = 4
    assert lib.rt_create(C.byref(g), 9, C.byref(o), 1e9, z.ctypes.data, z.ctypes.data,
                         np.ones(1).ctypes.data, C.byref(h)) == R.RT_EINVAL
    assert lib.rt_create(C.byref(g), 1, C.byref(o), -1.0, z.ctypes.data, z.ctypes.data,
                         np.ones(1).ctypes.data, C.byref(h)) == R.RT_EINVAL
    g.bc[0] = R.RT_BC_PERIODIC   # periodic on one face only
    assert lib.rt_create(C.byref(g), 1, C.byref(o), 1e9, z.ctypes.data, z.ctypes.data,
                         np.ones(1).ctypes.data, C.byref(h)) == R.RT_EINVAL
    assert lib.rt_step(None, 0.0) == R.RT_EINVAL
    assert lib.rt_last_error(None) == b"null handle"


def test_hll_table_matches_oracle_table(lib):
    """The library's closed-form wave speeds against the oracle's own table
    (complex-step Jacobian + LAPACK eigenvalues)."""
    from oracle import hll_table as H
    from paper_1304_7126_gb300 import rt as R
    a = R.rt_hll_table(257, 257)
    b = H.table()
    assert np.max(np.abs(a - b)) < 1e-12


def test_noalloc_rejects_what_rt_create_rejects(lib):
    """rt_thermo_step_noalloc checks its options and constants like
    rt_create (finite c_r, dt and a_exp, finite non-negative cross sections,
    finite positive energies) before any CUDA call; the device pointers are
    never touched on these paths."""
    from paper_1304_7126_gb300 import rt as R
    o = R.default_options()
    sig = np.array([[1e-18, 0.0, 0.0]])
    egy = np.array([3e-11])
    fake = [C.c_void_p(256) for _ in range(8)]   # stand-ins for device arrays, never dereferenced

    def call(cr=3e9, dt=1e12, sN=sig, sE=sig, e=egy, opt=o, n=1):
        return lib.rt_thermo_step_noalloc(C.c_longlong(n), 1, C.byref(opt), C.c_double(cr), sN.ctypes.data,
                                          sE.ctypes.data, e.ctypes.data, C.c_double(dt), *fake, None)

    lib.rt_thermo_step_noalloc.restype = C.c_int
    inf, nan = float("inf"), float("nan")
    assert call(cr=inf) == R.RT_EINVAL
    assert call(cr=0.0) == R.RT_EINVAL
    assert call(dt=inf) == R.RT_EINVAL
    assert call(dt=nan) == R.RT_EINVAL
    assert call(sN=np.array([[inf, 0.0, 0.0]])) == R.RT_EINVAL
    assert call(sE=np.array([[1e-18, nan, 0.0]])) == R.RT_EINVAL
    assert call(e=np.array([0.0])) == R.RT_EINVAL
    assert call(e=np.array([inf])) == R.RT_EINVAL
    assert call(n=0) == R.RT_EINVAL
    assert call(n=262145) == R.RT_EINVAL
    bad = R.default_options(a_exp=inf)
    assert call(opt=bad) == R.RT_EINVAL


def test_adjoint_contract_matches_its_checks():
    """The header's contract for rt_step_vjp names what the argument check in
    rt_api.cu rejects (precision, OTSA, smoothing) and both fluxes, since the
    check accepts either."""
    hdr = open(os.path.join(ROOT, "include", "rt.h")).read()
    block = hdr[hdr.index("---- adjoint"):hdr.index("int rt_step_vjp")]
    api = open(os.path.join(ROOT, "paper_1304_7126_gb300", "csrc", "rt_api.cu")).read()
    check = api[api.index("int vjp_args"):]
    check = check[:check.index("\n}\n")]
    assert "opt.flux" not in check       # either flux is accepted ...
    assert "RT_GLF" in block and "RT_HLL" in block   # ... and the header says so
    for word, cond in (("RT_FP64", "precision != RT_FP64"), ("OTSA", "!h->opt.otsa"), ("smooth", "opt.smooth")):
        assert cond in check and word in block, word


def test_routing_entry_point_rejects_null(lib):
    assert lib.rt_set_thermo_routing(None, 1, 2, 3, 0) == -1

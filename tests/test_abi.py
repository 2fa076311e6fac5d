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

"""Algorithmic operation counts of the RT step (test and measurement
infrastructure).

``opcount.cpp`` compiles the oracle's own source (``rt_oracle.c``) as C++
with every double replaced by a counting scalar of the same layout, so the
counts are those of the method as the oracle states it (Sec. 3.2 transport,
App. A thermochemistry), not of the CUDA library's arrangement of it.
:func:`counting` swaps that build in for the oracle inside a ``with``
block; the oracle's Python API (``oracle.Problem`` ...) is unchanged.

Counted per operation: additions and subtractions, multiplications,
divisions and square roots (one flop each); calls of exp, log and pow are
counted apart.  ``make_counts.py`` writes the per-unit figures the
benchmark reports its roofline against.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess

from . import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "opcount.cpp")
LIB = os.path.join(HERE, "liboracle_ops.so")
FIELDS = ("add", "mul", "div", "sqrt", "exp", "log", "pow")
_lib = None


def build(force: bool = False) -> str:
    deps = [SRC, O.SRC, os.path.join(HERE, "rt_oracle.h")]
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(d) for d in deps):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp,
                               SRC, "-lm"], cwd=HERE)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = O.bind(C.CDLL(LIB))
        L.oracle_opcount_get.argtypes = [C.POINTER(C.c_ulonglong)]
        L.oracle_opcount_reset.argtypes = []
        _lib = L
    return _lib


def reset():
    lib().oracle_opcount_reset()


def counts() -> dict:
    a = (C.c_ulonglong * 7)()
    lib().oracle_opcount_get(a)
    d = dict(zip(FIELDS, (int(v) for v in a)))
    d["flop"] = d["add"] + d["mul"] + d["div"] + d["sqrt"]
    return d


@contextlib.contextmanager
def counting():
    """Run the oracle's Python API on the counting build (single-threaded:
    the counters are plain globals) with the counters reset on entry."""
    saved = O._lib
    O._lib = lib()
    reset()
    try:
        yield
    finally:
        O._lib = saved

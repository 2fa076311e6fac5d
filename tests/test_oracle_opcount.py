"""The op-counting build of the oracle (oracle/opcount.cpp): it runs the
oracle's own code, so its results are the oracle's bits, and its counts
follow the arithmetic as written (hand counts of small functions)."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def OC():
    from oracle import opcount
    opcount.build()
    return opcount


def test_same_bits_as_the_oracle(oracle_mod, OC):
    from paper_1304_7126_gb300 import workloads as W
    w = W.small_cosmo(6, seed=3, nsrc=1)
    p = oracle_mod.Problem(w.shape, w.dx, w.G, w.cr, w.sigN, w.sigE, w.egy, X=w.X, flux=w.flux, bc=w.bc)
    dt = oracle_mod.courant_dt(w.cfl, w.dx, w.cr)
    a, b = w.state(), w.state()
    ra = p.step(a, dt, w.src_ijk, w.src_L)
    with OC.counting():
        rb = p.step(b, dt, w.src_ijk, w.src_L)
        c = OC.counts()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(ra[2], rb[2])
    assert c["flop"] > 0 and c["exp"] > 0


def test_hand_counts(oracle_mod, OC):
    with OC.counting():
        oracle_mod.chi(0.3)   # (3 + 4 f f) / (5 + 2 sqrt(4 - 3 f f))
        c = OC.counts()
    assert (c["add"], c["mul"], c["div"], c["sqrt"]) == (3, 5, 1, 1)
    with OC.counting():
        oracle_mod.courant_dt(0.8, 1e20, 3e9)   # cfl dx / (3 c_r)
        c = OC.counts()
    assert (c["add"], c["mul"], c["div"], c["sqrt"], c["flop"]) == (0, 2, 1, 0, 3)

"""Batched boxes (rt_batch_*) against single-box handles and the oracle.

Each box of a batch runs the same arithmetic as a single handle on the same
box (same closure, face fluxes and update per cell; the thermochemistry is
per cell), so the states must agree bit for bit whatever the tiling the
autotuner picks; the per-box budgets agree to rounding."""
import numpy as np
import pytest

from parity import compare, oracle_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_1304_7126_gb300 import rt
    rt.load()
    return rt


def _boxes(flux, n=7):
    from paper_1304_7126_gb300 import workloads as W
    return W.batched(n, seed0=77, steps=6, sides=(8, 12, 16, 20, 33), flux=flux)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("flux", [1, 0])
def test_batch_equals_single_boxes(R, prec, flux):
    p = {"fp64": R.RT_FP64, "mixed": R.RT_MIXED}[prec]
    boxes = _boxes(flux)
    assert len({b.G for b in boxes}) == 2 and len({b.shape for b in boxes}) > 2
    bt = R.RTBatch.from_workloads(boxes, precision=p)
    dt = bt.courant_dt()
    bt.run(dt, 3)
    bt.autotune(1)
    bt.step(dt)
    bt.run(dt, 2)
    for i, w in enumerate(boxes):
        single = R.RT.from_workload(w, precision=p)
        single.run(dt, 6)
        a, b = single.get_state(), bt.get_box_state(i)
        for k in a:
            assert np.array_equal(a[k], b[k]), (i, k)
        ba, bb = single.budget(), bt.budget(i)
        assert np.allclose(ba, bb, rtol=1e-12, atol=1e-12 * ba[:, 3:4].max())
        single.close()


def test_batch_both_tile_shapes_in_one_launch(R):
    """Boxes of side 32 take the 32 x 8 tiles and the others 16 x 16 (the
    default shapes), so one step's single transport launch runs CTAs of
    both: every box still equals its single-box run bit for bit."""
    from paper_1304_7126_gb300 import workloads as W
    boxes = W.batched(3, seed0=77, steps=3, sides=(32,), flux=1) + W.batched(3, seed0=90, steps=3, sides=(20,), flux=1)
    bt = R.RTBatch.from_workloads(boxes)
    shapes = []
    for i in range(len(boxes)):
        sh, _ = bt.tiling(i)
        shapes.append(sh)
    assert set(shapes) == {0, 1}, shapes
    dt = bt.courant_dt()
    bt.run(dt, 3)
    for i, w in enumerate(boxes):
        single = R.RT.from_workload(w)
        single.run(dt, 3)
        a, b = single.get_state(), bt.get_box_state(i)
        for k in a:
            assert np.array_equal(a[k], b[k]), (i, k)
        single.close()


def test_batch_box_vs_oracle(oracle_mod, R):
    boxes = _boxes(1, n=4)
    bt = R.RTBatch.from_workloads(boxes)
    dt = bt.courant_dt()
    bt.run(dt, 4)
    for i in (0, 3):
        w = boxes[i]
        p = oracle_problem(oracle_mod, w, nthreads=4)
        ref = w.state()
        for _ in range(4):
            st, _, _, _ = p.step(ref, dt, w.src_ijk, w.src_L)
            assert st == 0
        e = compare(bt.get_box_state(i), ref, cr=w.cr, G=w.G)
        assert max(e.values()) < 1e-10, (i, e)
    b = bt.budget(0)
    resid = b[:, 3] - b[:, 0] - b[:, 1] - b[:, 2]
    in0 = 0.0   # boxes start without photons
    assert np.all(np.abs(resid - in0) <= 1e-12 * b[:, 3])


def test_batch_rejects_bad_boxes(R):
    from paper_1304_7126_gb300 import workloads as W
    boxes = _boxes(1, n=2)
    boxes[1].dx = boxes[0].dx * 1.5
    with pytest.raises(R.RTError):
        R.RTBatch(boxes)

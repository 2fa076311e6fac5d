"""The double-float exp, log, log1p, reciprocal and square root of the FP64
rate fits (dfmath.cuh: float pairs on the FP32 pipe, Tang's table-driven
reductions) against CUDA's FP64 functions (torch's CUDA exp, log, log1p,
reciprocal, sqrt) over random arguments across the whole range each is used
on, within the stated bounds (doubles outside 2^-60 .. 2^60 in magnitude
take CUDA's own function):
  exp(x)     relative (3 |x| + 16) 2^-48  (the argument is a 48-bit pair; its low
             float and the reduction each round once)
  log(x)     absolute 2^-46 max(1, |ln x|)
  log1p(w)   relative 2^-45
  1/a, sqrt  relative 2^-44
  softplus   absolute 2^-45 max(1, |x|), its derivative absolute 2^-42
exact at the special points (exp 0 = 1, log 1 = 0, underflow to 0,
overflow to infinity)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TINY = 2.0 ** -1074


@pytest.fixture(scope="module")
def R():
    import torch
    assert torch.cuda.is_available()
    from paper_1304_7126_gb300 import rt
    rt.load()
    return rt


def _eval(R, fn, x):
    import torch
    xd = torch.as_tensor(x, dtype=torch.float64).cuda()
    y = torch.empty_like(xd)
    rc = R.load().rt_fmath_eval(fn, xd.numel(), xd.data_ptr(), y.data_ptr(), None)
    assert rc == 0
    torch.cuda.synchronize()
    return xd, y


def _check(got, ref, bound):
    got, ref = got.cpu().numpy(), ref.cpu().numpy()
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    err = np.abs(got[fin] - ref[fin])
    q = err / np.maximum(bound[fin], 4 * TINY)
    return float(q.max()) if q.size else 0.0


def test_exp(R):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-745.0, 709.7, 400000), rng.uniform(-40.0, 40.0, 200000),
                        np.sign(rng.standard_normal(100000)) * 10 ** rng.uniform(-300, 0, 100000),
                        [0.0, -0.0, 1e-320, -708.39, -708.4, -744.0, -745.0, 709.78, -750.0, 710.0]])
    xd, y = _eval(R, 0, x)
    ref = xd.exp()
    bound = ref.abs().cpu().numpy() * ((3 * np.abs(x) + 16) * 2.0 ** -48)
    assert _check(y, ref, bound) <= 1.0
    yc = y.cpu().numpy()
    assert yc[-10] == 1.0 and yc[-9] == 1.0 and yc[-2] == 0.0 and np.isinf(yc[-1])


def test_log(R):
    rng = np.random.default_rng(2)
    x = np.concatenate([10 ** rng.uniform(-307, 308, 400000), 1.0 + rng.uniform(-1e-3, 1e-3, 200000),
                        rng.uniform(0.5, 2.0, 200000), 10 ** rng.uniform(0, 10, 200000),
                        [1.0, 2.0, 0.5, 5e-324, 1e-310, 2.2250738585072014e-308, 1.7976931348623157e308]])
    xd, y = _eval(R, 1, x)
    ref = xd.log()
    bound = np.maximum(1.0, np.abs(ref.cpu().numpy())) * 2.0 ** -46
    assert _check(y, ref, bound) <= 1.0
    assert y.cpu().numpy()[-7] == 0.0


def test_log1p(R):
    rng = np.random.default_rng(3)
    w = np.concatenate([10 ** rng.uniform(-300, 300, 400000), rng.uniform(0.0, 4.0, 200000),
                        rng.uniform(0.0, 0.05, 200000), 10 ** rng.uniform(-20, -10, 100000),
                        [0.0, 1e-300, 1e-17, 1.0, 1e300, 0.03125]])
    wd, y = _eval(R, 2, w)
    ref = wd.log1p()
    bound = ref.abs().cpu().numpy() * 2.0 ** -45
    assert _check(y, ref, bound) <= 1.0


@pytest.mark.parametrize("fn", [3, 4])
def test_reciprocal_and_sqrt(R, fn):
    rng = np.random.default_rng(4 + fn)
    x = np.concatenate([10 ** rng.uniform(-300, 300, 300000), 10 ** rng.uniform(0, 10, 300000),
                        rng.uniform(0.5, 2.0, 100000), [1.0, 4.0, 1e-310, 1e308]])
    xd, y = _eval(R, fn, x)
    ref = xd.reciprocal() if fn == 3 else xd.sqrt()
    bound = ref.abs().cpu().numpy() * 2.0 ** -44
    assert _check(y, ref, bound) <= 1.0


def test_softplus_and_derivative(R):
    import torch
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.uniform(-16.0, 16.0, 400000), rng.uniform(-1.0, 1.0, 100000),
                        np.arange(-16.0, 16.0, 0.25), [-30.0, -16.0001, 15.9999, 16.0, 25.0]])
    xd, y = _eval(R, 5, x)
    ref = torch.nn.functional.softplus(xd, threshold=1000.0)
    bound = np.maximum(1.0, np.abs(x)) * 2.0 ** -45
    assert _check(y, ref, bound) <= 1.0
    _, s = _eval(R, 6, x)
    sref = torch.sigmoid(xd)
    assert _check(s, sref, np.full(x.shape, 2.0 ** -42)) <= 1.0


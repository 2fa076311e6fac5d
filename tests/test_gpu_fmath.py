"""The table-driven FP64 exp, log and log1p of the rate fits (fmath.cuh,
Tang's methods) against CUDA's own functions (torch's CUDA exp, log,
log1p), in units in the last place of the CUDA result: at most 2 ulp over
random arguments across the whole range each is used on (including
subnormal results and inputs), exact at the special points."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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


def _ulps(got, ref):
    got, ref = got.cpu().numpy(), ref.cpu().numpy()
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    d = np.abs(got[fin] - ref[fin]) / np.spacing(np.abs(ref[fin]))
    return float(d.max()) if d.size else 0.0


def test_exp(R):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(-745.0, 709.7, 400000), rng.uniform(-40.0, 40.0, 200000),
                        np.sign(rng.standard_normal(100000)) * 10 ** rng.uniform(-300, 0, 100000),
                        [0.0, -0.0, 1e-320, -708.39, -708.4, -744.0, -745.0, 709.78, -750.0, 710.0]])
    xd, y = _eval(R, 0, x)
    assert _ulps(y, xd.exp()) <= 2.0
    yc = y.cpu().numpy()
    assert yc[-10] == 1.0 and yc[-9] == 1.0 and yc[-2] == 0.0 and np.isinf(yc[-1])


def test_log(R):
    rng = np.random.default_rng(2)
    x = np.concatenate([10 ** rng.uniform(-307, 308, 400000), 1.0 + rng.uniform(-1e-3, 1e-3, 200000),
                        rng.uniform(0.5, 2.0, 200000), [1.0, 2.0, 0.5, 5e-324, 1e-310, 2.2250738585072014e-308,
                                                         1.7976931348623157e308]])
    xd, y = _eval(R, 1, x)
    assert _ulps(y, xd.log()) <= 2.0
    assert y.cpu().numpy()[-7] == 0.0


def test_log1p(R):
    rng = np.random.default_rng(3)
    w = np.concatenate([10 ** rng.uniform(-300, 300, 400000), rng.uniform(0.0, 4.0, 200000),
                        10 ** rng.uniform(-20, -10, 100000), [0.0, 1e-300, 1e-17, 1.0, 1e300]])
    wd, y = _eval(R, 2, w)
    assert _ulps(y, wd.log1p()) <= 2.0

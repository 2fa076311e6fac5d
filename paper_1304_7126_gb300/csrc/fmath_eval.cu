// rt_fmath_eval: the double-float exp, log, log1p, reciprocal, square root,
// and softplus with its derivative of dfmath.cuh (the ones the FP64
// thermochemistry uses) over a device array of doubles, so
// that their accuracy can be checked against CUDA's own; rt_rate_functions:
// the rate-function table of rates.cuh, for host-side checks.
#include <cuda_runtime.h>

#include "dfmath.cuh"
#include "rates.cuh"
#include "rt.h"

namespace rtgb {
namespace {

__device__ double eval_one(int fn, double v)
{
    using namespace dfm;
    switch (fn) {
    case 0: return splittable(v) ? exp2d(split(v)) : exp(v);
    case 1: return to_double(logd(v));
    case 2: return (v >= 0.0 && !splittable(v)) ? log1p(v) : to_double(log1pd(v));
    case 3: return (v > 0.0 && splittable(v)) ? to_double(rcp(split(v))) : 1.0 / v;
    case 4: return (v > 0.0 && splittable(v)) ? to_double(sqrt2(split(v))) : sqrt(v);
    case 5: {   // ln(1 + e^v)
        double sg;
        return to_double(softplus2(split_any(v), sg));
    }
    default: {   // 1 / (1 + e^-v)
        double sg;
        softplus2(split_any(v), sg);
        return sg;
    }
    }
}

__global__ void fmath_kernel(int fn, long long n, const double *__restrict__ x, double *__restrict__ y)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = eval_one(fn, x[i]);
}

}  // namespace
}  // namespace rtgb

extern "C" int rt_fmath_eval(int fn, long long n, const double *x, double *y, void *stream)
{
    if (fn < 0 || fn > 6 || n < 0 || (n > 0 && (!x || !y))) return RT_EINVAL;
    if (n == 0) return RT_OK;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    rtgb::fmath_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(fn, n, x, y);
    if (cudaGetLastError() != cudaSuccess) return RT_ECUDA;
    return RT_OK;
}

extern "C" int rt_rate_functions(int case_b, double *out)
{
    using namespace rtgb;
    if ((case_b != 0 && case_b != 1) || !out) return RT_EINVAL;
    static constexpr RateFnTab tab[2] = {make_rate_fns(0), make_rate_fns(1)};
    auto d = [](dfm::F2 v) { return (double)v.hi + (double)v.lo; };
    for (int k = 0; k < 32; ++k) {
        const RateFn &q = tab[case_b].f[k];
        double *o = out + 7 * k;
        o[0] = q.Cc;
        o[1] = d(q.c0);
        o[2] = d(q.c1);
        o[3] = d(q.c2);
        o[4] = d(q.c3);
        o[5] = d(q.c4);
        o[6] = d(q.c5);
    }
    return RT_OK;
}

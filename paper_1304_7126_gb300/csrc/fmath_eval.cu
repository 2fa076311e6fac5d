// rt_fmath_eval: the table-driven exp, log and log1p of fmath.cuh over a
// device array, so that their accuracy can be checked against CUDA's own.
#include <cuda_runtime.h>

#include "fmath.cuh"
#include "rt.h"

namespace rtgb {
namespace {

__global__ void fmath_kernel(int fn, long long n, const double *__restrict__ x, double *__restrict__ y)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double v = x[i];
        y[i] = fn == 0 ? fm::exp_t(v) : (fn == 1 ? fm::log_t(v) : fm::log1p_t(v));
    }
}

}  // namespace
}  // namespace rtgb

extern "C" int rt_fmath_eval(int fn, long long n, const double *x, double *y, void *stream)
{
    if (fn < 0 || fn > 2 || n < 0 || (n > 0 && (!x || !y))) return RT_EINVAL;
    if (n == 0) return RT_OK;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    rtgb::fmath_kernel<<<(unsigned)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(fn, n, x, y);
    if (cudaGetLastError() != cudaSuccess) return RT_ECUDA;
    return RT_OK;
}

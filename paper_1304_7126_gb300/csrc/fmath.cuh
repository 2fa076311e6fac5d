// Table-driven FP64 exp, log and log1p for the rate transcendentals.
//
// On GB300 a dependent FP64 instruction has 64 cycles of latency, and the
// rate fits of one temperature form a chain log -> exp -> log1p -> exp that
// the longest-sub-cycling cells run thousands of times per RT step.  These
// follow P. T. P. Tang's table-driven methods (exp: ACM TOMS 15 (1989) 144;
// log: ACM TOMS 16 (1990) 378) with short polynomials evaluated in Estrin
// form, so that each function is a chain of about eight dependent FP64
// operations.  Their error is within a few units in the last place
// (checked against CUDA's exp, log and log1p by tests/test_gpu_fmath.py);
// the tables and split constants come from gen_fmath_tables.py.
//
// exp:   x = (32 m + j) ln2/32 + r, |r| <= ln2/64, reduced with a two-part
//        ln2/32; exp(x) = 2^m 2^(j/32) (1 + p(r)), p the Taylor polynomial
//        of e^r - 1 to degree 6 (truncation < 4e-18 relative).
// log:   x = 2^e m, m in [1, 2), F = 1 + j/128 nearest m, f = m - F
//        (exact), u = f / F with a tabulated 1/F, |u| <= 1/256;
//        ln x = e ln2 + ln F + q(u), q the Taylor polynomial of ln(1 + u)
//        to degree 7 (truncation < 1e-20).
// log1p: v = 1 + w rounded; ln(1 + w) = ln v + (w - (v - 1)) / v.
#pragma once

#include <cuda_runtime.h>

#include "fmath_tables.h"

namespace rtgb {
namespace fm {

__device__ __forceinline__ double exp_t(double x)
{
    if (!(x > -745.2)) return (x != x) ? x : 0.0;   // NaN passes, underflow to 0
    if (x > 709.79) return __longlong_as_double(0x7ff0000000000000LL);
    const double nd = rint(x * kFmInvLn2x32);
    const int n = (int)nd;
    double r = fma(-nd, kFmLn2d32Hi, x);
    r = fma(-nd, kFmLn2d32Lo, r);
    const int j = n & 31;
    const int m = n >> 5;   // floor(n / 32)
    const double r2 = r * r;
    const double a = fma(r, 1.0 / 6.0, 0.5);
    const double b = fma(r2, 1.0 / 720.0, fma(r, 1.0 / 120.0, 1.0 / 24.0));
    const double q = fma(r2, b, a);
    const double p = fma(r2, q, r);   // e^r - 1
    const double t = __ldg(&kFmExp2Tab[j]);
    const double y = fma(t, p, t);
    if (m > -1022 && m < 1024) return y * __hiloint2double((m + 1023) << 20, 0);
    return ldexp(y, m);
}

__device__ __forceinline__ double log_t(double x)
{
    if (!(x > 0.0) || x == __longlong_as_double(0x7ff0000000000000LL)) {
        if (x == 0.0) return -__longlong_as_double(0x7ff0000000000000LL);
        return (x > 0.0) ? x : __longlong_as_double(0x7ff8000000000000LL);
    }
    int hi = __double2hiint(x);
    int lo = __double2loint(x);
    int e = (hi >> 20) - 1023;
    if (e == -1023) {   // subnormal: scale by 2^54 first
        const double xs = x * 18014398509481984.0;
        hi = __double2hiint(xs);
        lo = __double2loint(xs);
        e = (hi >> 20) - 1023 - 54;
    }
    const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);   // [1, 2)
    const int j = (int)((m - 1.0) * 128.0 + 0.5);
    const double F = 1.0 + (double)j * (1.0 / 128.0);
    const double f = m - F;
    const double u = f * __ldg(&kFmLogTab[j][0]);
    const double u2 = u * u;
    const double a = fma(u, 1.0 / 3.0, -0.5);
    const double b = fma(u, 0.2, -0.25);
    const double c = fma(u, 1.0 / 7.0, -1.0 / 6.0);
    const double u4 = u2 * u2;
    const double q = fma(u4, c, fma(u2, b, a));
    const double p = fma(u2, q, u);   // ln(1 + u)
    const double ed = (double)e;
    const double head = fma(ed, kFmLn2Hi, __ldg(&kFmLogTab[j][1]));
    const double tail = fma(ed, kFmLn2Lo, __ldg(&kFmLogTab[j][2]));
    return head + (p + tail);
}

__device__ __forceinline__ double log1p_t(double w)
{
    const double v = 1.0 + w;
    if (v == 1.0) return w;
    const double c = w - (v - 1.0);
    return log_t(v) + c * (double)__frcp_rn((float)v);
}

}  // namespace fm
}  // namespace rtgb

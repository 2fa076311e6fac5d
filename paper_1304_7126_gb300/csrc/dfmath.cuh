// Double-float ("F2") exp, log, log1p, square root and reciprocal for the
// rate transcendentals, on the FP32 pipe.
//
// On GB300 a warp issues one FP64 instruction per ~64 cycles whatever the
// dependences between them (one FP64 FMA chain and two independent chains
// per warp both run at 64 cycles per FMA), while a dependent FP32 FMA takes
// ~4.6 cycles; float <-> double conversions also run on the FP64 pipe.  A
// thermochemistry attempt is therefore bounded by its count of FP64
// instructions, and the transcendentals of the rate fits were about half
// of them.  Here every value is an unevaluated sum hi + lo of two floats
// (48 significant bits, the double-float arithmetic of Dekker, Numer. Math.
// 18 (1971) 224, with the error-free sum of Knuth and the FMA product);
// doubles enter and leave through integer bit operations, and each result
// costs one FP64 addition (hi + lo, exact).  exp and log follow P. T. P.
// Tang's table-driven reductions (ACM TOMS 15 (1989) 144 and 16 (1990)
// 378) with 64 and 128 table points; the tables and split constants come
// from gen_dfmath_tables.py.
//
// Accuracy (relative to the exact function of the double input, checked
// against CUDA's FP64 exp, log and log1p by tests/test_gpu_fmath.py):
//   exp(x)    (3 |x| + 16) 2^-48 (the 48-bit argument dominates for |x| > 8)
//   log(x)    2^-46 max(1, |ln x|) absolute
//   log1p(w)  2^-45
//   1/a, sqrt(a) of a pair: 2^-44
// i.e. 1e-14 to 1e-12 relative for the rate coefficients, far inside the
// 1e-10 parity the FP64 path is held to.  Inputs outside the ranges the
// rate fits produce (a double beyond 2^-60 .. 2^60 in magnitude) go to
// CUDA's FP64 functions (log1p of w < 2^-60 is w itself).
#pragma once

#include <cuda_runtime.h>

#include "dfmath_tables.h"

namespace rtgb {
namespace dfm {

struct F2 {
    float hi, lo;   // value hi + lo, |lo| <= ulp(hi) / 2
};

// ---- error-free transformations (rounded intrinsics: never contracted) ----
__device__ __forceinline__ F2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ F2 fast_two_sum(float a, float b)   // |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ F2 two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// ---- double-float arithmetic ----
__device__ __forceinline__ F2 add(F2 a, F2 b)
{
    F2 s = two_sum(a.hi, b.hi);
    const F2 t = two_sum(a.lo, b.lo);
    s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ F2 add(F2 a, float b)
{
    const F2 s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ F2 neg(F2 a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ F2 mul(F2 a, F2 b)
{
    F2 p = two_prod(a.hi, b.hi);
    p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
    p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ F2 mul(F2 a, float b)
{
    F2 p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}

// 2^n as a float, n in [-126, 127]
__device__ __forceinline__ float pow2f(int n) { return __uint_as_float((unsigned)(n + 127) << 23); }

// ---- doubles in and out through integer operations ----
// |x| in [2^-60, 2^60) (or 0): the double split into a float pair (hi: the
// top 24 bits, lo: the next 29 rounded to 24), relative error <= 2^-48; the
// range keeps the low floats of the results below (reciprocals, square
// roots, logarithms) clear of float subnormals.
__device__ __forceinline__ bool splittable(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffULL;
    return b == 0ULL || (b >= 0x3c30000000000000ULL && b < 0x43b0000000000000ULL);
}

__device__ __forceinline__ F2 split(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return {0.0f, 0.0f};
    if (e == 0x7ff) return {__uint_as_float(sign | 0x7f800000u | ((b & 0xfffffffffffffULL) ? 0x400000u : 0u)), 0.0f};
    const float hi = __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7fffff));
    const float lo = __uint2float_rn((unsigned)(b & 0x1fffffffULL)) * pow2f(e - 1075);
    return {hi, sign ? -lo : lo};
}

// any double as a pair (outside the range above through FP64 conversions)
__device__ __forceinline__ F2 split_any(double x)
{
    if (splittable(x)) return split(x);
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - (double)hi)};
}

// the double of a float (exact; subnormal floats, which the pairs here never
// hold in a significant place, count as zero)
__device__ __forceinline__ double widen(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xff;
    if (e == 0) return 0.0;
    const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) |
                                    ((unsigned long long)(e + 896) << 52) |
                                    ((unsigned long long)(u & 0x7fffff) << 29);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double to_double(F2 a) { return widen(a.hi) + widen(a.lo); }

// 1 / a and sqrt(a) of a positive pair: one Newton step in pair arithmetic
// from the correctly rounded FP32 value (relative error <= 2^-24, squared by
// the step)
__device__ __forceinline__ F2 rcp(F2 a)
{
    const float r0 = __frcp_rn(a.hi);
    const F2 e = two_prod(a.hi, r0);
    const float err = __fsub_rn(__fsub_rn(1.0f, e.hi), __fmaf_rn(a.lo, r0, e.lo));
    return fast_two_sum(r0, r0 * err);
}

// 1/a refined by a second Newton step in pair arithmetic (2^-47)
__device__ __forceinline__ F2 rcp2(F2 a)
{
    const F2 r = rcp(a);
    const F2 e = add(F2{1.0f, 0.0f}, neg(mul(a, r)));
    return add(r, mul(r, e));
}

__device__ __forceinline__ F2 sqrt2(F2 a)
{
    const float s0 = __fsqrt_rn(a.hi);
    const F2 p = two_prod(s0, s0);
    const float d = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo);
    return fast_two_sum(s0, d * rsqrtf(a.hi) * 0.5f);
}

// ---- elementary functions ----
// exp2d, log2f2 and log1pd are called out of line: inlined at every call
// site of every thermochemistry kernel they made ptxas run for tens of
// minutes.  The warp path of the rates (one call site per temperature)
// inlines exp2d_inl and log2f2_inl, the same arithmetic.

// e^x of a pair; a double result (subnormal, 0 and infinity as CUDA's exp)
__device__ __forceinline__ double exp2d_inl(F2 x)
{
    if (!(x.hi > -745.2f)) return (x.hi != x.hi) ? (double)x.hi : 0.0;
    if (x.hi > 709.78f) return __longlong_as_double(0x7ff0000000000000LL);
    const float kf = rintf(__fmul_rn(x.hi, kDfInvL));
    const int k = (int)kf;
    // r = x - k ln2/64: k L1 exact, x.hi - k L1 exact (Sterbenz), k L2 split
    // exactly; x.lo, the low part of k L2 and k L3 (all below 2^-24 |x|)
    // summed in FP32
    const F2 p2 = two_prod(kf, kDfL2);
    const F2 s = two_sum(__fmaf_rn(-kf, kDfL1, x.hi), -p2.hi);
    const F2 r = fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(x.lo, __fmaf_rn(kf, kDfL3, p2.lo))));
    // e^r - 1 = r + [r^2/2 + r^3 (1/6 + r/24 + r^2/120)], |r| <= ln2/128; the
    // bracket (< 1.6e-5) as a pair from r.hi^2 exactly plus FP32 terms
    const float rh = r.hi;
    const F2 h2 = two_prod(rh, rh);
    const float c = __fmaf_rn(rh, r.lo,
                              rh * h2.hi * __fmaf_rn(rh, __fmaf_rn(rh, 1.0f / 120.0f, 1.0f / 24.0f), 1.0f / 6.0f));
    const F2 q = fast_two_sum(0.5f * h2.hi, __fmaf_rn(0.5f, h2.lo, c));
    const F2 p = add(r, q);
    const float2 t = __ldg(&kDfExp2Tab[k & 63]);
    const F2 T{t.x, t.y};
    const F2 y = add(T, mul(T, p));   // 2^(j/64) e^r
    const double yd = to_double(y);
    const int m = k >> 6;              // floor(k / 64)
    if (m > -1020 && m < 1020)
        return __longlong_as_double(__double_as_longlong(yd) + ((long long)m << 52));
    return ldexp(yd, m);
}

static __device__ __noinline__ double exp2d(F2 x) { return exp2d_inl(x); }

// ln of a positive normal pair
__device__ __forceinline__ F2 log2f2_inl(F2 v)
{
    const unsigned bits = __float_as_uint(v.hi);
    const int e = (int)(bits >> 23) - 127;
    const int j = (int)(((bits & 0x7fffff) + (1u << 15)) >> 16);   // F = 1 + j/128 nearest the mantissa
    const float Fs = __uint_as_float((unsigned)(e + 127) << 23) * (1.0f + (float)j * (1.0f / 128.0f));
    // f = v - F 2^e: exact (Sterbenz), then scaled exactly to v / 2^e - F
    const F2 fs = two_sum(__fsub_rn(v.hi, Fs), v.lo);
    const float sc = pow2f(-e);
    const F2 f{fs.hi * sc, fs.lo * sc};
    const float4 L = __ldg(&kDfLogTab[j]);
    const F2 u = mul(f, F2{L.z, L.w});   // u = f / F, |u| <= 1/256
    // ln(1 + u) = u - u^2/2 + u^3 (1/3 - u/4 + u^2/5 - u^3/6)
    const F2 u2 = mul(u, u);
    const F2 u3 = mul(u2, u.hi);
    const float uh = u.hi;
    const float cub = uh * __fmaf_rn(uh, __fmaf_rn(uh, -1.0f / 6.0f, 0.2f), -0.25f);
    F2 q = add(u, F2{-0.5f * u2.hi, -0.5f * u2.lo});
    q = add(q, mul(u3, F2{kDfThirdHi, kDfThirdLo}));
    q = add(q, u3.hi * cub);
    // e ln2 + ln F + q
    const float ef = (float)e;
    F2 s = two_prod(ef, kDfLn2B);
    s = add(F2{ef * kDfLn2A, 0.0f}, s);   // e A exact
    s = add(s, ef * kDfLn2C);
    s = add(s, F2{L.x, L.y});
    return add(s, q);
}

static __device__ __noinline__ F2 log2f2(F2 v) { return log2f2_inl(v); }

// ln x of a double
__device__ __forceinline__ F2 logd(double x)
{
    if (x > 0.0 && splittable(x)) return log2f2(split(x));
    const double r = log(x);
    return split(r);   // out of range: CUDA's log, split (|ln x| < 746)
}

// ln(1 + w) of a double w >= 0
static __device__ __noinline__ F2 log1pd(double w)
{
    if (!(w >= 0.0) || w >= 1.152921504606847e18) return split(log1p(w));   // NaN, w >= 2^60
    if (!splittable(w)) return {__double2float_rn(w), 0.0f};                     // w < 2^-60: ln(1 + w) = w
    const F2 W = split(w);
    if (W.hi < 0.03125f) {
        // 2 atanh(z), z = w / (2 + w) <= 1/65: 2 (z + z^3/3 + z^5/5 + z^7/7)
        const F2 rd = rcp(add(W, 2.0f));   // 1 / (2 + w)
        const F2 z = mul(W, rd);
        const F2 z2 = mul(z, z);
        const float zh = z2.hi;
        F2 s = mul(z2, F2{kDfThirdHi, kDfThirdLo});
        s = add(s, zh * zh * __fmaf_rn(zh, 1.0f / 7.0f, 0.2f));
        const F2 y = add(z, mul(z, s));
        return {2.0f * y.hi, 2.0f * y.lo};
    }
    // v = 1 + w exactly as a pair plus a remainder c below its last bit
    const F2 s = two_sum(1.0f, W.hi);
    const F2 t = two_sum(s.lo, W.lo);
    const F2 v = fast_two_sum(s.hi, t.hi);
    const F2 lv = log2f2(v);
    return add(lv, __fdividef(t.lo, v.hi));   // + c / v
}

// ln(1 + e^z) of a pair z, with its derivative 1/(1 + e^-z) as a double.
// On [-16, 16): the interpolating polynomials of kDfSoftplusTab (degree 9
// in t = z - middle of a 1/4-wide interval, |t| <= 1/8); the terms of
// degree 5 and up are below 2^-24 of the value, so they are summed in
// FP32, the rest in pair arithmetic (absolute error ~1e-14 at |z| ~ 16,
// that of the pair coefficients).  Outside (temperatures far beyond the
// fits' range) from e^z and log1p.
__device__ __forceinline__ F2 softplus2(F2 z, double &sig)
{
    if (z.hi >= (float)kDfSpLo && z.hi < -(float)kDfSpLo) {
        int k = (int)__fmul_rn(__fadd_rn(z.hi, -(float)kDfSpLo), (float)kDfSpPer);
        k = k < kDfSpN - 1 ? k : kDfSpN - 1;
        const float mid = (float)kDfSpLo + ((float)k + 0.5f) / (float)kDfSpPer;   // exact
        const F2 t = add(z, -mid);
        const float th = t.hi;
        const float2 *c = kDfSoftplusTab[k];
        float r = __ldg(&c[9].x), q = 9.0f * r;
        r = __fmaf_rn(r, th, __ldg(&c[8].x));
        q = __fmaf_rn(q, th, 8.0f * __ldg(&c[8].x));
        r = __fmaf_rn(r, th, __ldg(&c[7].x));
        q = __fmaf_rn(q, th, 7.0f * __ldg(&c[7].x));
        r = __fmaf_rn(r, th, __ldg(&c[6].x));
        q = __fmaf_rn(q, th, 6.0f * __ldg(&c[6].x));
        r = __fmaf_rn(r, th, __ldg(&c[5].x));
        q = __fmaf_rn(q, th, 5.0f * __ldg(&c[5].x));
        F2 P{r, 0.0f}, D{q, 0.0f};
#pragma unroll
        for (int n = 4; n >= 0; --n) {
            const float2 cn = __ldg(&c[n]);
            P = add(F2{cn.x, cn.y}, mul(P, t));
            if (n >= 1) D = add(mul(F2{cn.x, cn.y}, (float)n), mul(D, t));
        }
        sig = to_double(D);
        return P;
    }
    const double w = exp2d(z);
    sig = w / (1.0 + w);
    return log1pd(w);
}

}  // namespace dfm
}  // namespace rtgb

// Device rate-coefficient fits of the paper's appendix on interaction rate
// coefficients (collisional ionisation: Cen 1992; recombination and
// recombination cooling: Hui & Gnedin 1997; collisional excitation: Cen
// 1992; bremsstrahlung; Compton: Haiman et al. 1996; dielectronic: Black
// 1981), each with its analytic temperature derivative, in FP64.
//
// Evaluation is split in two stages so that the same arithmetic can be done
// by one thread or spread over the lanes of a warp:
//   1. transcendentals of one temperature (struct Transc; exp, log, log1p,
//      square root and reciprocal in the double-float arithmetic of
//      dfmath.cuh, on the FP32 pipe): ln T, sqrt T,
//      1/T, and twelve exponentials exp(a ln T + b/T + c) - the Boltzmann
//      factors exp(-T0/T), the power laws, and w = (lam/l0)^r of the four
//      Hui & Gnedin fits A lam^p / (1 + w)^s - then log1p(w) and
//      exp(p ln lam - s log1p(w)) of those four fits;
//   2. assembly of the rates and derivatives from Transc (plain arithmetic).
// transc_serial computes stage 1 in one thread; transc_warp lets lane k of a
// warp evaluate exponential k, so a warp pays for three exponential levels
// instead of twenty transcendental calls.  Both use identical expressions,
// so they give identical bits.
#pragma once

#include <cuda_runtime.h>

#include "dual.cuh"
#include "dfmath.cuh"

namespace rtgb {

// Quotients of the thermochemistry (IEEE division; a double-float quotient
// refined by an FP64 residual step was tried and its longer dependent chain
// made every attempt slower)
template <typename S>
__device__ __forceinline__ S qdiv(const S &a, const S &b) { return a / b; }

// exp arguments: exp(fma(a, ln T, fma(b, 1/T, c)))
enum {
    E_BETA_HI = 0,   // exp(-157809.1/T): beta_HI, zeta_HI
    E_BETA_HEI,      // exp(-285335.4/T): beta_HeI, zeta_HeI
    E_BETA_HEII,     // exp(-631515/T):   beta_HeII, zeta_HeII
    E_PSI_HI,        // exp(-118348/T)
    E_PSI_HEII,      // T^-0.397 exp(-473638/T)
    E_OMEGA1,        // T^-1.5 exp(-470000/T)
    E_OMEGA2,        // exp(-94000/T)
    E_ALPHA_HEII,    // (570670/T)^p
    E_W0,            // w = exp(z) of the Hui & Gnedin fits HG_* (their z = ln w
                     // are the arguments E_W0.. of the table; w itself is not formed)
    NEXP = E_W0 + 4
};
enum { HG_ALPHA_HII = 0, HG_ALPHA_HEIII, HG_ETA_HII, HG_ETA_HEIII, NHG };

struct ExpArg {
    double a, b, c;
};
struct HGPar {
    double A, lnT1, p, r, s;   // A lam^p / (1 + w)^s, lam = T1/T, w = (lam/l0)^r
};
struct RateTable {           // one per recombination case (A, B)
    ExpArg ea[NEXP];
    HGPar hg[NHG];
    double A_aHeII, p_aHeII;  // alpha_HeII = A (570670/T)^p
};

// S: double, or Dual (dual.cuh) when the adjoint differentiates the rates
template <typename S>
struct TranscT {
    S lnT, sqrtT, invT, u;   // u = 1 / (1 + sqrt(T / 1e5))
    S e[NEXP];
    S l[NHG];                 // log1p(w) = softplus(z), z = ln w
    S s[NHG];                 // w / (1 + w), the derivative of softplus at z
    S v[NHG];                 // exp(p ln lam - s log1p(w))
};
using Transc = TranscT<double>;

// Rate tables: exp(a ln T + b/T + c) arguments and the Hui &
// Gnedin parameters, case A then case B; the logarithms are of the fits'
// temperature constants and pivots.
#define RTGB_RATE_TAB_INIT {\
    { /* case A */ \
        {{0.0, -157809.1, 0.0}, {0.0, -285335.4, 0.0}, {0.0, -631515.0, 0.0}, {0.0, -118348.0, 0.0}, {-0.397, -473638.0, 0.0}, {-1.5, -470000.0, 0.0}, {0.0, -94000.0, 0.0}, {-0.654, 0.0, 8.668486417830579}, {-0.47, 0.0, 6.2568105714688285}, {-0.47, 0.0, 6.908582567206}, {-0.502, 0.0, 6.664858835981581}, {-0.502, 0.0, 7.361006797385964}},\
        {{1.269e-13, 12.662275226919286, 1.503, 0.47, 1.923}, {2.538e-13, 14.049024154019651, 1.503, 0.47, 1.923}, {1.778e-29, 12.662275226919286, 1.965, 0.502, 2.697}, {1.4224e-28, 14.049024154019651, 1.965, 0.502, 2.697}},\
        3e-14, 0.654 },\
    { /* case B */ \
        {{0.0, -157809.1, 0.0}, {0.0, -285335.4, 0.0}, {0.0, -631515.0, 0.0}, {0.0, -118348.0, 0.0}, {-0.397, -473638.0, 0.0}, {-1.5, -470000.0, 0.0}, {0.0, -94000.0, 0.0}, {-0.75, 0.0, 9.940924791090113}, {-0.407, 0.0, 4.743307143753357}, {-0.407, 0.0, 5.307713957083206}, {-0.376, 0.0, 4.456105724024312}, {-0.376, 0.0, 4.977523320614049}},\
        {{2.753e-14, 12.662275226919286, 1.5, 0.407, 2.242}, {5.506e-14, 14.049024154019651, 1.5, 0.407, 2.242}, {3.435e-30, 12.662275226919286, 1.97, 0.376, 3.72}, {2.748e-29, 14.049024154019651, 1.97, 0.376, 3.72}},\
        1.26e-14, 0.75 }\
}
// uniform reads (an index the same in every lane): the constant cache
static __constant__ RateTable c_rate_tab[2] = RTGB_RATE_TAB_INIT;
// lane-indexed reads (lane k evaluates term k): global memory through the
// L1 cache, which serves different addresses of a warp in one request where
// the constant cache would serialise them
static __device__ const RateTable g_rate_tab[2] = RTGB_RATE_TAB_INIT;
// compile-time copy, for the derived constants of the cooling terms
constexpr RateTable kRateTabCx[2] = RTGB_RATE_TAB_INIT;
#undef RTGB_RATE_TAB_INIT

// The table's constants as float pairs (hi = the double rounded to a float,
// lo = the rest rounded), made at compile time: a ln T + b/T + c and
// p (ln T1 - ln T) - s l in pair arithmetic without splitting doubles at
// run time.
struct RateTableF2 {
    dfm::F2 ea[NEXP][3];   // a, b, c
    dfm::F2 hg[NHG][3];    // ln T1, p, s
};
constexpr dfm::F2 pair_of(double x)
{
    return dfm::F2{(float)x, (float)(x - (double)(float)x)};
}
constexpr RateTableF2 make_rate_f2(int cb)
{
    RateTableF2 t{};
    const RateTable &R = kRateTabCx[cb];
    for (int k = 0; k < NEXP; ++k) {
        t.ea[k][0] = pair_of(R.ea[k].a);
        t.ea[k][1] = pair_of(R.ea[k].b);
        t.ea[k][2] = pair_of(R.ea[k].c);
    }
    for (int j = 0; j < NHG; ++j) {
        t.hg[j][0] = pair_of(R.hg[j].lnT1);
        t.hg[j][1] = pair_of(R.hg[j].p);
        t.hg[j][2] = pair_of(R.hg[j].s);
    }
    return t;
}
static __device__ const RateTableF2 g_rate_f2[2] = {make_rate_f2(0), make_rate_f2(1)};

__device__ __forceinline__ dfm::F2 ldg2(const dfm::F2 &v)
{
    const float2 f = __ldg(reinterpret_cast<const float2 *>(&v));
    return dfm::F2{f.x, f.y};
}

// a ln T + b / T + c of table entry k
__device__ __forceinline__ dfm::F2 exp_arg2(const RateTableF2 &R, int k, dfm::F2 lnT, dfm::F2 invT)
{
    using namespace dfm;
    return add(add(ldg2(R.ea[k][2]), mul(lnT, ldg2(R.ea[k][0]))), mul(invT, ldg2(R.ea[k][1])));
}

// p (ln T1 - ln T) - s l of Hui & Gnedin fit j
__device__ __forceinline__ dfm::F2 hg_arg2(const RateTableF2 &R, int j, dfm::F2 lnT, dfm::F2 l)
{
    using namespace dfm;
    return add(mul(add(ldg2(R.hg[j][0]), neg(lnT)), ldg2(R.hg[j][1])), neg(mul(l, ldg2(R.hg[j][2]))));
}

// Stage 1 in double-float arithmetic (dfmath.cuh): ln T, 1/T, sqrt T and u
// as float pairs, each exponential's argument formed in pair arithmetic and
// e^x returned as a double; the Transc values are the doubles of the pairs.
constexpr double kUc = 0.003162277660168379;   // 1 / sqrt(1e5)
constexpr float kUcHi = (float)kUc;
constexpr float kUcLo = (float)(kUc - (double)kUcHi);

__device__ __forceinline__ void transc_level0(double T, Transc &t, dfm::F2 &lnT, dfm::F2 &invT)
{
    using namespace dfm;
    if (!(T > 0.0) || !splittable(T)) {   // not reached by T >= 1 K below 2^120 K
        t.lnT = log(T);
        t.sqrtT = sqrt(T);
        t.invT = 1.0 / T;
        t.u = 1.0 / (1.0 + t.sqrtT * kUc);
        lnT = split_any(t.lnT);
        invT = split_any(t.invT);
        return;
    }
    const F2 T2 = split(T);
    lnT = log2f2(T2);
    invT = rcp(T2);
    const F2 sq = sqrt2(T2);
    const F2 u = rcp(add(mul(sq, F2{kUcHi, kUcLo}), 1.0f));
    t.lnT = to_double(lnT);
    t.sqrtT = to_double(sq);
    t.invT = to_double(invT);
    t.u = to_double(u);
}

// Stage 1 in one thread.  need: bit k of the exponentials E_*, bit NEXP + j
// of the Hui & Gnedin fits j.  A Hui & Gnedin fit A lam^p / (1 + w)^s with
// w = (lam/l0)^r is exp(p ln lam - s softplus(z)), z = r ln(lam/l0): one
// polynomial for ln(1 + e^z) (dfm::softplus2) instead of an exp and a log1p.
__device__ __forceinline__ void transc_serial(double T, int case_b, unsigned need, Transc &t)
{
    const RateTableF2 &R = g_rate_f2[case_b];
    dfm::F2 lnT, invT;
    transc_level0(T, t, lnT, invT);
#pragma unroll
    for (int k = 0; k < E_W0; ++k)
        if (need & (1u << k)) t.e[k] = dfm::exp2d(exp_arg2(R, k, lnT, invT));
#pragma unroll
    for (int j = 0; j < NHG; ++j) {
        if (need & (1u << (NEXP + j))) {
            double sg;
            const dfm::F2 l = dfm::softplus2(exp_arg2(R, E_W0 + j, lnT, invT), sg);
            t.l[j] = dfm::to_double(l);
            t.s[j] = sg;
            t.v[j] = dfm::exp2d(hg_arg2(R, j, lnT, l));
        }
    }
}

// Stage 1 spread over a full warp (all 32 lanes must call it with the same
// T); every lane ends with the complete, identical Transc.  Lanes 0..7
// take the exponentials, lanes 8..11 the Hui & Gnedin fits, and every lane
// runs the same instructions (a warp runs divergent paths one after the
// other): the exponential lanes pass z = 0 through the softplus and ignore
// it, then all lanes take one exp of their argument.
__device__ __forceinline__ void transc_warp(double T, int case_b, Transc &t)
{
    const RateTableF2 &R = g_rate_f2[case_b];
    const int lane = threadIdx.x & 31;
    dfm::F2 lnT, invT;
    transc_level0(T, t, lnT, invT);
    const bool fit = lane >= E_W0 && lane < E_W0 + NHG;
    const int j = (lane - E_W0) & 3;
    const dfm::F2 arg = exp_arg2(R, lane < E_W0 ? lane : E_W0 + j, lnT, invT);
    double sj;
    const dfm::F2 l = dfm::softplus2(fit ? arg : dfm::F2{0.0f, 0.0f}, sj);
    const dfm::F2 hga = hg_arg2(R, j, lnT, l);
    const double ek = dfm::exp2d(fit ? hga : arg);
    const double lj = dfm::to_double(l);
#pragma unroll
    for (int q = 0; q < E_W0; ++q) t.e[q] = __shfl_sync(0xffffffffu, ek, q);
#pragma unroll
    for (int q = 0; q < NHG; ++q) {
        t.l[q] = __shfl_sync(0xffffffffu, lj, E_W0 + q);
        t.s[q] = __shfl_sync(0xffffffffu, sj, E_W0 + q);
        t.v[q] = __shfl_sync(0xffffffffu, ek, E_W0 + q);
    }
}

// FP32 transcendentals (the mixed-precision thermochemistry): the same
// arguments evaluated in single precision, stored widened into Transc so the
// assembly below is shared (widened through integer operations: a float ->
// double conversion would take the FP64 pipe; float subnormals, far below
// any rate that matters, count as zero).  Relative accuracy ~1e-7.
// a double rounded to the nearest float (ties away from zero) through
// integer operations: a double -> float conversion would take the FP64
// pipe.  Below the normal float range the result is 0, above it infinity
// (NaN included).  Truncating instead biases the FP32 absorption
// coefficients by half an ulp, which over a source cell's thousands of
// sub-steps moved the mixed-precision results by 1e-4.
__device__ __forceinline__ float narrow(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const unsigned long long a = (b & 0x7fffffffffffffffULL) + 0x10000000ULL;   // carry may raise the exponent
    const int e = (int)(a >> 52);
    if (e < 897) return __uint_as_float(sign);
    if (e > 1150) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((unsigned)(e - 896) << 23) | (unsigned)((a >> 29) & 0x7fffff));
}

__device__ __forceinline__ void transc_level0_f(double T, Transc &t, float &lnT, float &invT)
{
    float Tf = narrow(T);
    lnT = logf(Tf);
    float sq = sqrtf(Tf);
    invT = 1.0f / Tf;
    t.lnT = dfm::widen(lnT);
    t.sqrtT = dfm::widen(sq);
    t.invT = dfm::widen(invT);
    t.u = dfm::widen(1.0f / (1.0f + sq * 0.0031622776f));
}

__device__ __forceinline__ float exp_arg_f(const ExpArg &q, float lnT, float invT)
{
    return fmaf(narrow(q.a), lnT, fmaf(narrow(q.b), invT, narrow(q.c)));
}

__device__ __forceinline__ float hg_arg_f(const HGPar &h, float lnT, float l)
{
    return narrow(h.p) * (narrow(h.lnT1) - lnT) - narrow(h.s) * l;
}

__device__ __forceinline__ void transc_serial_f(double T, int case_b, unsigned need, Transc &t)
{
    const RateTable &R = c_rate_tab[case_b];
    float lnT, invT;
    transc_level0_f(T, t, lnT, invT);
#pragma unroll
    for (int k = 0; k < E_W0; ++k)
        if (need & (1u << k)) t.e[k] = dfm::widen(expf(exp_arg_f(R.ea[k], lnT, invT)));
#pragma unroll
    for (int j = 0; j < NHG; ++j) {
        if (need & (1u << (NEXP + j))) {
            const float w = expf(exp_arg_f(R.ea[E_W0 + j], lnT, invT));
            const float l = log1pf(w);
            t.l[j] = dfm::widen(l);
            t.s[j] = dfm::widen(w / (1.0f + w));
            t.v[j] = dfm::widen(expf(hg_arg_f(R.hg[j], lnT, l)));
        }
    }
}

__device__ __forceinline__ void transc_warp_f(double T, int case_b, Transc &t)
{
    const RateTable &R = g_rate_tab[case_b];
    const int lane = threadIdx.x & 31;
    float lnT, invT;
    transc_level0_f(T, t, lnT, invT);
    float ek, lj = 0.0f, sj = 0.0f;
    if (lane < E_W0) {
        ek = expf(exp_arg_f(R.ea[lane], lnT, invT));
    } else {
        const int j = (lane - E_W0) & 3;
        const float w = expf(exp_arg_f(R.ea[E_W0 + j], lnT, invT));
        lj = log1pf(w);
        sj = w / (1.0f + w);
        ek = expf(hg_arg_f(R.hg[j], lnT, lj));
    }
#pragma unroll
    for (int q = 0; q < E_W0; ++q) t.e[q] = dfm::widen(__shfl_sync(0xffffffffu, ek, q));
#pragma unroll
    for (int q = 0; q < NHG; ++q) {
        t.l[q] = dfm::widen(__shfl_sync(0xffffffffu, lj, E_W0 + q));
        t.s[q] = dfm::widen(__shfl_sync(0xffffffffu, sj, E_W0 + q));
        t.v[q] = dfm::widen(__shfl_sync(0xffffffffu, ek, E_W0 + q));
    }
}

// Stage 1 for a dual temperature: values from transc_serial (so they are
// the bits of the double path), derivatives by the chain rule:
// d lnT = dT/T, d sqrtT = sqrtT dT/(2T), d(1/T) = -dT/T^2, du = -u^2 k d sqrtT,
// d exp(a lnT + b/T + c) = e (a d lnT + b d(1/T)), d softplus(z) = sigma dz,
// d exp(p (lnT1 - lnT) - s l) = v (-p d lnT - s dl).
__device__ __forceinline__ void transc_dual(const Dual &T, int case_b, unsigned need, TranscT<Dual> &t)
{
    const RateTable &R = c_rate_tab[case_b];
    Transc p;
    transc_serial(T.v, case_b, need, p);
    const double dT = T.d;
    const double dln = p.invT * dT, dinv = -p.invT * p.invT * dT;
    const double dsq = 0.5 * p.sqrtT * p.invT * dT;
    t.lnT = Dual(p.lnT, dln);
    t.sqrtT = Dual(p.sqrtT, dsq);
    t.invT = Dual(p.invT, dinv);
    t.u = Dual(p.u, -p.u * p.u * 0.003162277660168379 * dsq);
#pragma unroll
    for (int k = 0; k < E_W0; ++k)
        if (need & (1u << k)) t.e[k] = Dual(p.e[k], p.e[k] * (R.ea[k].a * dln + R.ea[k].b * dinv));
#pragma unroll
    for (int j = 0; j < NHG; ++j) {
        if (need & (1u << (NEXP + j))) {
            // z = a lnT + b/T + c; d softplus(z) = sigma dz, d sigma = sigma (1 - sigma) dz
            const double dz = R.ea[E_W0 + j].a * dln + R.ea[E_W0 + j].b * dinv;
            const double sg = p.s[j];
            const double dl = sg * dz;
            t.l[j] = Dual(p.l[j], dl);
            t.s[j] = Dual(sg, sg * (1.0 - sg) * dz);
            t.v[j] = Dual(p.v[j], p.v[j] * (-R.hg[j].p * dln - R.hg[j].s * dl));
        }
    }
}

// d ln v / dT of a Hui & Gnedin fit: -(1/T) (p - s r w / (1 + w))
template <typename S>
__device__ __forceinline__ S hg_dlog(const HGPar &h, const TranscT<S> &t, int j)
{
    return -t.invT * (h.p - h.s * h.r * t.s[j]);
}

// bits of Transc needed by each consumer
constexpr unsigned kNeedH = (1u << E_BETA_HI) | (1u << E_W0) | (1u << (NEXP + HG_ALPHA_HII));
constexpr unsigned kNeedHe = (1u << E_BETA_HEI) | (1u << E_BETA_HEII) | (1u << E_ALPHA_HEII) |
                             (1u << (E_W0 + HG_ALPHA_HEIII)) | (1u << (NEXP + HG_ALPHA_HEIII));
constexpr unsigned kNeedHe3 = (1u << E_BETA_HEII) | (1u << (E_W0 + HG_ALPHA_HEIII)) |
                              (1u << (NEXP + HG_ALPHA_HEIII));
constexpr unsigned kNeedCoolH = (1u << E_BETA_HI) | (1u << E_PSI_HI) | (1u << (E_W0 + HG_ETA_HII)) |
                                (1u << (NEXP + HG_ETA_HII));
// the three recombination rates alpha_HII, alpha_HeII, alpha_HeIII
constexpr unsigned kNeedRec = (1u << E_ALPHA_HEII) | (1u << (E_W0 + HG_ALPHA_HII)) |
                              (1u << (E_W0 + HG_ALPHA_HEIII)) | (1u << (NEXP + HG_ALPHA_HII)) |
                              (1u << (NEXP + HG_ALPHA_HEIII));
constexpr unsigned kNeedCoolHe = (1u << E_BETA_HEI) | (1u << E_BETA_HEII) | (1u << E_PSI_HEII) |
                                 (1u << E_OMEGA1) | (1u << E_OMEGA2) | (1u << E_ALPHA_HEII) |
                                 (1u << (E_W0 + HG_ETA_HEIII)) | (1u << (NEXP + HG_ETA_HEIII));

template <typename S>
struct HRatesT {      // rates needed by the x_HII update
    S beta, dbeta, alpha, dalpha;
};
template <typename S>
struct HeRatesT {
    S beta_HeI, beta_HeII, alpha_HeII, alpha_HeIII;
};
using HRates = HRatesT<double>;
using HeRates = HeRatesT<double>;

// Cen (1992) form A sqrt(T) u exp(-T0/T)
template <typename S>
__device__ __forceinline__ void cen_fit(double A, double T0, const S &e, const TranscT<S> &t, S &v, S &dv)
{
    v = A * t.sqrtT * t.u * e;
    dv = v * (0.5 * t.u * t.invT + T0 * t.invT * t.invT);
}

template <typename S>
__device__ __forceinline__ void h_rates_from(const TranscT<S> &t, int case_b, HRatesT<S> &r)
{
    const RateTable &R = c_rate_tab[case_b];
    cen_fit(5.85e-11, 157809.1, t.e[E_BETA_HI], t, r.beta, r.dbeta);
    r.alpha = R.hg[HG_ALPHA_HII].A * t.v[HG_ALPHA_HII];
    r.dalpha = r.alpha * hg_dlog(R.hg[HG_ALPHA_HII], t, HG_ALPHA_HII);
}

template <typename S>
__device__ __forceinline__ void he_rates_from(const TranscT<S> &t, int case_b, HeRatesT<S> &r)
{
    const RateTable &R = c_rate_tab[case_b];
    S d;
    cen_fit(2.38e-11, 285335.4, t.e[E_BETA_HEI], t, r.beta_HeI, d);
    cen_fit(5.68e-12, 631515.0, t.e[E_BETA_HEII], t, r.beta_HeII, d);
    r.alpha_HeII = R.A_aHeII * t.e[E_ALPHA_HEII];
    r.alpha_HeIII = R.hg[HG_ALPHA_HEIII].A * t.v[HG_ALPHA_HEIII];
}

// Recombination rates of HII, HeII, HeIII (the case of the table t was
// evaluated with)
template <typename S>
__device__ __forceinline__ void recomb_alphas(const TranscT<S> &t, int case_b, S a[3])
{
    const RateTable &R = c_rate_tab[case_b];
    a[0] = R.hg[HG_ALPHA_HII].A * t.v[HG_ALPHA_HII];
    a[1] = R.A_aHeII * t.e[E_ALPHA_HEII];
    a[2] = R.hg[HG_ALPHA_HEIII].A * t.v[HG_ALPHA_HEIII];
}

// Primordial cooling magnitude L (Eq. (rate_cooling), positive = cooling)
// and dL/dT, as a sum of terms of one form,
//     C n_s sqrt(T)^a u^b T^c X1 X2 A,
// X1 an exponential e[i1] of the Transc (or the Hui & Gnedin value v[hg]),
// X2 an optional second exponential, A the fit's amplitude where the rate
// table holds it (it depends on the recombination case), n_s a density;
// each term's T-derivative is the term times its log-derivative
//     a/(2T) - b (1 - u)/(2T) + c/T + dln X1/dT + dln X2/dT,
// dln e/dT = a_e/T - b_e/T^2 from the exponential's argument, and the Hui &
// Gnedin log-derivative.  The terms (collisional ionisation and excitation,
// recombination and dielectronic cooling, bremsstrahlung) are summed in a
// fixed pairwise order; Compton cooling is added after.  All products and
// sums are rounded as written (rmul, radd), so the one-thread sum and the
// warp sum (lane k evaluates term k) give the same bits.
enum { SP_HI = 0, SP_HII, SP_HEI, SP_HEII, SP_HEIII, SP_FF, NSP };   // SP_FF: n_HII + n_HeII + 4 n_HeIII

struct CoolTerm {
    double C;
    int sq, uu, tt;   // powers (0 or 1) of sqrt T, u, T
    int e1, e2, hg;   // exponentials e[e1], e[e2] and Hui & Gnedin fit hg (-1: none)
    int amp;          // 1: times the table's amplitude of alpha_HeII
    int sp;           // density factor SP_*
    int he;           // a helium term
};

// (the paper's fits: Cen 1992 collisional ionisation and excitation, Hui &
// Gnedin 1997 recombination cooling, Black 1981 dielectronic recombination,
// bremsstrahlung; k_B T alpha_HeII for HeII recombination cooling)
#define RTGB_COOL_TERMS(X)                                                           \
    X(1.27e-21, 1, 1, 0, E_BETA_HI, -1, -1, 0, SP_HI, 0)                              \
    X(7.5e-19, 0, 1, 0, E_PSI_HI, -1, -1, 0, SP_HI, 0)                                \
    X(1.0, 0, 0, 1, -1, -1, HG_ETA_HII, 0, SP_HII, 0)                                 \
    X(1.42e-27, 1, 0, 0, -1, -1, -1, 0, SP_FF, 0)                                     \
    X(9.38e-22, 1, 1, 0, E_BETA_HEI, -1, -1, 0, SP_HEI, 1)                            \
    X(4.95e-22, 1, 1, 0, E_BETA_HEII, -1, -1, 0, SP_HEII, 1)                          \
    X(5.54e-17, 0, 1, 0, E_PSI_HEII, -1, -1, 0, SP_HEII, 1)                           \
    X(1.380649e-16, 0, 0, 1, E_ALPHA_HEII, -1, -1, 1, SP_HEII, 1)                     \
    X(1.24e-13, 0, 0, 0, E_OMEGA1, -1, -1, 0, SP_HEII, 1)                             \
    X(0.3 * 1.24e-13, 0, 0, 0, E_OMEGA1, E_OMEGA2, -1, 0, SP_HEII, 1)                 \
    X(1.0, 0, 0, 1, -1, -1, HG_ETA_HEIII, 0, SP_HEIII, 1)
#define RTGB_COOL_ROW(C, a, b, c, e1, e2, hg, amp, sp, he) {C, a, b, c, e1, e2, hg, amp, sp, he},
constexpr int kNCool = 11;
// row k at compile time (the one-thread sum, unrolled)
__host__ __device__ __forceinline__ constexpr CoolTerm cool_row(int k)
{
    constexpr CoolTerm rows[kNCool] = {RTGB_COOL_TERMS(RTGB_COOL_ROW)};
    return rows[k];
}
// the same rows in device memory, indexed by lane (the warp sum)
static __device__ const CoolTerm kCoolTermsDev[kNCool] = {RTGB_COOL_TERMS(RTGB_COOL_ROW)};
#undef RTGB_COOL_ROW
#undef RTGB_COOL_TERMS

// a[i] through selects (registers, not local memory, for a lane-dependent
// i; a plain a[i] once unrolled with a constant i)
template <typename T, int N>
__device__ __forceinline__ T pick(const T (&a)[N], int i)
{
    T r = a[0];
#pragma unroll
    for (int j = 1; j < N; ++j) r = (i == j) ? a[j] : r;
    return r;
}

// dln e/dT of exp(a ln T + b/T + c)
template <typename S>
__device__ __forceinline__ S exp_dlog(const ExpArg &q, const S &x)
{
    return radd(rmul(x, q.a), rmul(rmul(x, x), -q.b));
}

// Per recombination case and term, the constants of the term and of its
// log-derivative, folded at compile time:
//   value  = Cc n_s sqrtT^sq u^uu T^tt X1 X2 v^hg, Cc = C (A_hg)^hg (A_aHeII)^amp
//   dln/dT = invT [K0 + U (1 - u) - Kb invT + SR sigma]
// with K0 = sq/2 + tt + a1 + a2 - hg p, U = -uu/2, Kb = b1 + b2,
// SR = hg s r (X_k = exp(a_k ln T + b_k / T + c_k), sigma = w/(1 + w) of
// the Hui & Gnedin fit: d ln v/dT = -(p - s r sigma)/T).
struct CoolK {
    double Cc, K0, U, Kb, SR;
};
struct CoolKTab {
    CoolK k[2][kNCool];
};
constexpr CoolKTab make_cool_k()
{
    CoolKTab t{};
    for (int cb = 0; cb < 2; ++cb) {
        const RateTable &R = kRateTabCx[cb];
        for (int k = 0; k < kNCool; ++k) {
            const CoolTerm q = cool_row(k);
            double Cc = q.C, K0 = 0.5 * q.sq + q.tt, Kb = 0.0, SR = 0.0;
            if (q.e1 >= 0) { K0 += R.ea[q.e1].a; Kb += R.ea[q.e1].b; }
            if (q.e2 >= 0) { K0 += R.ea[q.e2].a; Kb += R.ea[q.e2].b; }
            if (q.hg >= 0) { Cc *= R.hg[q.hg].A; K0 -= R.hg[q.hg].p; SR = R.hg[q.hg].s * R.hg[q.hg].r; }
            if (q.amp) Cc *= R.A_aHeII;
            t.k[cb][k] = CoolK{Cc, K0, -0.5 * q.uu, Kb, SR};
        }
    }
    return t;
}
static __device__ const CoolKTab g_cool_k = make_cool_k();

// One term and its T-derivative; q the row, kc its constants.  A factor the
// row lacks multiplies by 1 and a missing part of the log-derivative adds
// 0 (both exact), so the one-thread sum (q known at compile time) and the
// warp sum (q indexed by lane) give the same bits.
template <typename S>
__device__ __forceinline__ void cool_term(const CoolTerm &q, const CoolK &kc, const TranscT<S> &t, const S &T,
                                          const S (&n)[NSP], S &v, S &dv)
{
    const S x = t.invT;
    const int e1 = q.e1 >= 0 ? q.e1 : 0, e2 = q.e2 >= 0 ? q.e2 : 0, hg = q.hg >= 0 ? q.hg : 0;
    const S one(1.0);
    const S a = rmul(q.sq ? t.sqrtT : one, q.uu ? t.u : one);
    const S b = rmul(q.tt ? T : one, q.e1 >= 0 ? pick(t.e, e1) : one);
    const S c = rmul(q.e2 >= 0 ? pick(t.e, e2) : one, q.hg >= 0 ? pick(t.v, hg) : one);
    const S f = rmul(rmul(rmul(a, b), rmul(c, pick(n, q.sp))), kc.Cc);
    const S sg = q.hg >= 0 ? pick(t.s, hg) : S(0.0);
    const S d = rfma(kc.U, radd(one, -t.u), S(kc.K0));
    const S d2 = rfma(kc.SR, sg, rfma(-kc.Kb, x, d));
    v = f;
    dv = rmul(f, rmul(d2, x));
}

// the fixed pairwise order of a 16-lane butterfly (offsets 8, 4, 2, 1)
template <typename S>
__device__ __forceinline__ S tree_sum16(S a[16])
{
#pragma unroll
    for (int m = 8; m >= 1; m >>= 1) {
#pragma unroll
        for (int i = 0; i < m; ++i) a[i] = radd(a[i], a[i + m]);
    }
    return a[0];
}

template <typename S>
__device__ __forceinline__ void cool_densities(const S &nHI, const S &nHII, const S &nHeI, const S &nHeII,
                                               const S &nHeIII, S n[NSP])
{
    n[SP_HI] = nHI;
    n[SP_HII] = nHII;
    n[SP_HEI] = nHeI;
    n[SP_HEII] = nHeII;
    n[SP_HEIII] = nHeIII;
    n[SP_FF] = radd(radd(nHII, nHeII), rmul(nHeIII, 4.0));
}

// + Compton, varpi = comp (T - T_gamma), comp = 1.017e-37 T_gamma^4 and
// T_gamma = 2.727/a (ThermoParams::comp, ::tg); both sums times n_e
template <typename S>
__device__ __forceinline__ void cooling_close(double comp, double tg, const S &T, const S &ne, const S &Ls,
                                              const S &dLs, S &L, S &dL)
{
    const S vp = rmul(radd(T, S(-tg)), comp);
    L = rmul(ne, radd(Ls, vp));
    dL = rmul(ne, radd(dLs, S(comp)));
}

// one thread
template <typename S>
__device__ __forceinline__ void cooling_from(const TranscT<S> &t, int case_b, double comp, double tg, bool helium,
                                             const S &T, const S &ne, const S &nHI, const S &nHII, const S &nHeI,
                                             const S &nHeII, const S &nHeIII, S &L, S &dL)
{
    S n[NSP];
    cool_densities(nHI, nHII, nHeI, nHeII, nHeIII, n);
    S a[16], b[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        a[k] = S(0.0);
        b[k] = S(0.0);
    }
#pragma unroll
    for (int k = 0; k < kNCool; ++k) {
        const CoolTerm q = cool_row(k);
        if (helium || !q.he) cool_term(q, g_cool_k.k[case_b][k], t, T, n, a[k], b[k]);
    }
    const S Ls = tree_sum16(a), dLs = tree_sum16(b);
    cooling_close(comp, tg, T, ne, Ls, dLs, L, dL);
}

// a full warp (all 32 lanes, the same arguments): lane k < 11 evaluates
// term k, the sums run over shuffles in the same pairwise order
__device__ __forceinline__ void cooling_warp(const Transc &t, int case_b, double comp, double tg, bool helium,
                                             double T, double ne, double nHI, double nHII, double nHeI,
                                             double nHeII, double nHeIII, double &L, double &dL)
{
    double n[NSP];
    cool_densities(nHI, nHII, nHeI, nHeII, nHeIII, n);
    const int k = threadIdx.x & 15;
    const int kk = k < kNCool ? k : 0;
    const CoolTerm q = kCoolTermsDev[kk];
    double v, dv;
    cool_term(q, g_cool_k.k[case_b][kk], t, T, n, v, dv);
    if (k >= kNCool || (!helium && q.he)) v = dv = 0.0;
#pragma unroll
    for (int m = 8; m >= 1; m >>= 1) {
        v = radd(v, __shfl_xor_sync(0xffffffffu, v, m));
        dv = radd(dv, __shfl_xor_sync(0xffffffffu, dv, m));
    }
    cooling_close(comp, tg, T, ne, v, dv, L, dL);
}

}  // namespace rtgb

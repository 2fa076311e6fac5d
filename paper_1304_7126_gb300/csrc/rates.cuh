// Device rate-coefficient fits of the paper's appendix on interaction rate
// coefficients (collisional ionisation: Cen 1992; recombination and
// recombination cooling: Hui & Gnedin 1997; collisional excitation: Cen
// 1992; bremsstrahlung; Compton: Haiman et al. 1996; dielectronic: Black
// 1981), each with its analytic temperature derivative, in FP64.
//
// Every rate coefficient and every cooling term is one function of T of
// the form
//     f(T) = Cc exp(c0 + c1 ln T + c2 / T - c3 softplus(c4 ln T + c5)),
// softplus(z) = ln(1 + e^z) (see RateFn below).  A warp evaluates them all
// at once, lane k function k; one thread evaluates the ones it needs.  The
// argument is formed in the double-float arithmetic of dfmath.cuh (on the
// FP32 pipe), exponentiated by dfm::exp2d and scaled by Cc in FP64; both
// paths run the same expressions and so give identical bits.
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
// compile-time copy, from which the rate functions below are built
constexpr RateTable kRateTabCx[2] = RTGB_RATE_TAB_INIT;
#undef RTGB_RATE_TAB_INIT

// The table's constants as float pairs (hi = the double rounded to a float,
// lo = the rest rounded), made at compile time.
constexpr dfm::F2 pair_of(double x)
{
    return dfm::F2{(float)x, (float)(x - (double)(float)x)};
}

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
#undef RTGB_COOL_ROW
#undef RTGB_COOL_TERMS

// ---- rate functions ----
//   Cen (1992) collisional rates A sqrt(T) u exp(-T0/T), u = 1/(1 + sqrt(T/1e5)):
//     Cc = A, c1 = 1/2, c2 = -T0, c3 = 1, z = (ln T - ln 1e5)/2, since
//     ln u = -softplus(z);
//   Hui & Gnedin (1997) fits A lam^p / (1 + (lam/l0)^r)^s, lam = T1/T:
//     Cc = A, c0 = p ln T1, c1 = -p, c3 = s, z = r ln(lam/l0) (the table's
//     argument E_W0 + j: a = -r, c = r (ln T1 - ln l0));
//   alpha_HeII = A (570670/T)^p and the Boltzmann factors: c3 = 0;
//   a cooling term C n_s sqrt(T)^sq u^uu T^tt X1 X2 v^hg adds the exponents
//     of its factors (no term has both u and a Hui & Gnedin factor) and
//     times its density n_s after the function.
// d ln f/dT = (c1 - c2/T - c3 c4 sigma(z)) / T, sigma = e^z / (1 + e^z).
enum {
    RF_COOL0 = 0,                 // slots 0..10: the cooling terms; 11..15 zero
    RF_BETA_HI = 16, RF_ALPHA_HII, RF_BETA_HEI, RF_BETA_HEII, RF_ALPHA_HEII, RF_ALPHA_HEIII,
    NRF
};
static_assert(kNCool <= 16 && NRF <= 32, "function slots are warp lanes");

struct RateFn {
    double Cc;
    dfm::F2 c0, c1, c2, c3, c4, c5;
    double d1, d2, d34, d344;   // c1, c2, c3 c4, c3 c4^2 (log-derivative and its derivative)
    float g34;                  // c3 c4 as a float (FP32 path)
};
struct RateFnTab {
    RateFn f[32];
};

constexpr double kHalfLn1e5 = 5.756462732485114;   // ln(1e5) / 2

constexpr RateFn rate_fn(double Cc, double c0, double c1, double c2, double c3, double c4, double c5)
{
    return RateFn{Cc, pair_of(c0), pair_of(c1), pair_of(c2), pair_of(c3), pair_of(c4), pair_of(c5),
                  c1, c2, c3 * c4, c3 * c4 * c4, (float)(c3 * c4)};
}
constexpr RateFn cen_fn(double A, double T0) { return rate_fn(A, 0.0, 0.5, -T0, 1.0, 0.5, -kHalfLn1e5); }
constexpr RateFn hg_fn(const RateTable &R, int j)
{
    return rate_fn(R.hg[j].A, R.hg[j].p * R.hg[j].lnT1, -R.hg[j].p, 0.0, R.hg[j].s, R.ea[E_W0 + j].a,
                   R.ea[E_W0 + j].c);
}
constexpr RateFn cool_fn(const RateTable &R, const CoolTerm &q)
{
    double Cc = q.C, c0 = 0.0, c1 = 0.5 * q.sq + q.tt, c2 = 0.0, c3 = 0.0, c4 = 0.0, c5 = 0.0;
    if (q.e1 >= 0) { c0 += R.ea[q.e1].c; c1 += R.ea[q.e1].a; c2 += R.ea[q.e1].b; }
    if (q.e2 >= 0) { c0 += R.ea[q.e2].c; c1 += R.ea[q.e2].a; c2 += R.ea[q.e2].b; }
    if (q.hg >= 0) {
        Cc *= R.hg[q.hg].A;
        c0 += R.hg[q.hg].p * R.hg[q.hg].lnT1;
        c1 -= R.hg[q.hg].p;
        c3 = R.hg[q.hg].s;
        c4 = R.ea[E_W0 + q.hg].a;
        c5 = R.ea[E_W0 + q.hg].c;
    }
    if (q.uu) { c3 = 1.0; c4 = 0.5; c5 = -kHalfLn1e5; }
    if (q.amp) Cc *= R.A_aHeII;
    return rate_fn(Cc, c0, c1, c2, c3, c4, c5);
}
constexpr RateFnTab make_rate_fns(int cb)
{
    RateFnTab t{};
    const RateTable &R = kRateTabCx[cb];
    for (int k = 0; k < kNCool; ++k) t.f[RF_COOL0 + k] = cool_fn(R, cool_row(k));
    for (int k = kNCool; k < 16; ++k) t.f[k] = rate_fn(0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0);
    t.f[RF_BETA_HI] = cen_fn(5.85e-11, 157809.1);
    t.f[RF_ALPHA_HII] = hg_fn(R, HG_ALPHA_HII);
    t.f[RF_BETA_HEI] = cen_fn(2.38e-11, 285335.4);
    t.f[RF_BETA_HEII] = cen_fn(5.68e-12, 631515.0);
    t.f[RF_ALPHA_HEII] = rate_fn(R.A_aHeII, R.ea[E_ALPHA_HEII].c, R.ea[E_ALPHA_HEII].a, R.ea[E_ALPHA_HEII].b, 0.0,
                                 0.0, 0.0);
    t.f[RF_ALPHA_HEIII] = hg_fn(R, HG_ALPHA_HEIII);
    for (int k = NRF; k < 32; ++k) t.f[k] = rate_fn(0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0);
    return t;
}
// uniform reads (one thread, a compile-time slot): the constant cache;
// lane-indexed reads (a warp): global memory through the L1 cache, which
// serves different addresses of a warp in one request
static __constant__ RateFnTab c_rate_fn[2] = {make_rate_fns(0), make_rate_fns(1)};
static __device__ const RateFnTab g_rate_fn[2] = {make_rate_fns(0), make_rate_fns(1)};

// density factor and helium flag of each cooling slot
static __device__ const int g_cool_sp[16] = {SP_HI, SP_HI, SP_HII, SP_FF, SP_HEI, SP_HEII, SP_HEII, SP_HEII,
                                             SP_HEII, SP_HEII, SP_HEIII, 0, 0, 0, 0, 0};

// ln T and 1/T of one temperature as pairs, 1/T as a double (both paths:
// the FP32 one needs ln T and 1/T to better than a float, see rate_value_f)
struct TLevel {
    dfm::F2 lnT, invT;
    double invTd;
};
template <bool MIX, bool INL = false>
__device__ __forceinline__ void t_level(double T, TLevel &L)
{
    using namespace dfm;
    if (!(T > 0.0) || !splittable(T)) {   // not reached by T >= 1 K below 2^60 K
        L.invTd = 1.0 / T;
        L.lnT = split_any(log(T));
        L.invT = split_any(L.invTd);
    } else {
        const F2 T2 = split(T);
        L.lnT = INL ? log2f2_inl(T2) : log2f2(T2);
        L.invT = rcp(T2);
        L.invTd = to_double(L.invT);
    }
}
// the same from 1/T as a pair
template <bool MIX, bool INL = false>
__device__ __forceinline__ void t_level_inv(dfm::F2 invT, TLevel &L)
{
    using namespace dfm;
    L.invT = invT;
    L.invTd = to_double(invT);
    if (invT.hi > 0.0f && splittable(L.invTd)) L.lnT = neg(INL ? log2f2_inl(invT) : log2f2(invT));
    else L.lnT = split_any(-log(L.invTd));
}
// f(T) of one function given l = softplus(z); all FP64 products rounded as
// written
__device__ __forceinline__ double rate_from_l(const RateFn &q, const TLevel &L, dfm::F2 l)
{
    using namespace dfm;
    const F2 arg = add(add(add(q.c0, mul(L.lnT, q.c1)), mul(L.invT, q.c2)), neg(mul(l, q.c3)));
    return rmul(q.Cc, exp2d(arg));
}
__device__ __forceinline__ dfm::F2 rate_softplus(const RateFn &q, const TLevel &L, double &sig)
{
    using namespace dfm;
    return softplus2(add(mul(L.lnT, q.c4), q.c5), sig);
}
// f(T) of one function and sigma(z)
__device__ __forceinline__ double rate_value(const RateFn &q, const TLevel &L, double &sig)
{
    return rate_from_l(q, L, rate_softplus(q, L, sig));
}
// df/dT = f (c1 - c2/T - c3 c4 sigma) / T
__device__ __forceinline__ double rate_deriv(const RateFn &q, double invT, double f, double sig)
{
    return rmul(f, rmul(rfma(-q.d34, sig, rfma(-q.d2, invT, q.d1)), invT));
}

// FP32 (the mixed-precision thermochemistry, RT_MIXED32): the argument is
// still formed in pairs (it reaches |20-60|, where a float's rounding alone
// is 1e-6 of the rate, and over thousands of sub-steps that moved N by 2e-4
// of the FP64 result), but the softplus correction ln(1 + e^-|z|) < ln 2
// and the exponential run in FP32: e^arg = e^hi (1 + lo) with the float
// exp of the high part; the log-derivative in FP32.  Relative accuracy
// ~2e-7.
__device__ __forceinline__ void rate_value_f(const RateFn &q, const TLevel &L, double &f, double &df)
{
    using namespace dfm;
    const F2 z = add(mul(L.lnT, q.c4), q.c5);
    const float e = __expf(-fabsf(z.hi));
    const float sg = (z.hi >= 0.0f ? 1.0f : e) / (1.0f + e);
    const F2 l = add(z.hi >= 0.0f ? z : F2{0.0f, 0.0f}, log1pf(e));   // softplus = max(z, 0) + ln(1 + e^-|z|)
    const F2 arg = add(add(add(q.c0, mul(L.lnT, q.c1)), mul(L.invT, q.c2)), neg(mul(l, q.c3)));
    const double eh = widen(expf(arg.hi));
    f = rmul(q.Cc, rfma(eh, widen(arg.lo), eh));
    const float x = L.invT.hi;
    const float g = __fmul_rn(__fmaf_rn(-q.g34, sg, __fmaf_rn(-q.c2.hi, x, q.c1.hi)), x);
    df = rmul(f, widen(g));
}
// values (and derivatives) of several functions at one temperature
template <typename S>
struct RatesT {
    S f[NRF], df[NRF];
};
using Rates = RatesT<double>;

__host__ __device__ constexpr unsigned rf_bit(int k) { return 1u << k; }
constexpr unsigned kNeedH = rf_bit(RF_BETA_HI) | rf_bit(RF_ALPHA_HII);   // values and derivatives
constexpr unsigned kNeedHe = rf_bit(RF_BETA_HEI) | rf_bit(RF_BETA_HEII) | rf_bit(RF_ALPHA_HEII) |
                             rf_bit(RF_ALPHA_HEIII);
constexpr unsigned kNeedHe3 = rf_bit(RF_BETA_HEII) | rf_bit(RF_ALPHA_HEIII);
constexpr unsigned kNeedRec = rf_bit(RF_ALPHA_HII) | rf_bit(RF_ALPHA_HEII) | rf_bit(RF_ALPHA_HEIII);
__host__ __device__ constexpr unsigned cool_mask(int he)
{
    unsigned m = 0;
    for (int k = 0; k < kNCool; ++k)
        if (cool_row(k).he == he) m |= rf_bit(RF_COOL0 + k);
    return m;
}
constexpr unsigned kNeedCoolH = cool_mask(0), kNeedCoolHe = cool_mask(1);

// slots whose softplus is that of u (z = (ln T - ln 1e5)/2, the same in
// all of them) and slots without a softplus (c3 = 0: l and sigma enter
// multiplied by zero, exactly)
__host__ __device__ constexpr unsigned rf_u_mask()
{
    unsigned m = rf_bit(RF_BETA_HI) | rf_bit(RF_BETA_HEI) | rf_bit(RF_BETA_HEII);
    for (int k = 0; k < kNCool; ++k)
        if (cool_row(k).uu) m |= rf_bit(RF_COOL0 + k);
    return m;
}
__host__ __device__ constexpr unsigned rf_plain_mask()
{
    unsigned m = rf_bit(RF_ALPHA_HEII);
    for (int k = 0; k < 16; ++k)
        if (k >= kNCool || (!cool_row(k).uu && cool_row(k).hg < 0)) m |= rf_bit(RF_COOL0 + k);
    return m;
}

// one thread: the functions in needF (derivatives of those in needD); the
// shared softplus of u once, none where it is multiplied by zero (the same
// bits as the warp, which evaluates every slot's own)
__device__ __forceinline__ void rates_serial(const TLevel &L, int case_b, unsigned needF, unsigned needD, Rates &r)
{
    constexpr unsigned kU = rf_u_mask(), kPlain = rf_plain_mask();
    const RateFnTab &R = c_rate_fn[case_b];
    double sgu = 0.0;
    dfm::F2 lu{0.0f, 0.0f};
    if (needF & kU) lu = rate_softplus(R.f[RF_BETA_HI], L, sgu);
#pragma unroll
    for (int k = 0; k < NRF; ++k) {
        if (needF & rf_bit(k)) {
            double sg = 0.0;
            if (kU & rf_bit(k)) {
                sg = sgu;
                r.f[k] = rate_from_l(R.f[k], L, lu);
            } else if (kPlain & rf_bit(k)) {
                r.f[k] = rate_from_l(R.f[k], L, dfm::F2{0.0f, 0.0f});
            } else {
                r.f[k] = rate_value(R.f[k], L, sg);
            }
            if (needD & rf_bit(k)) r.df[k] = rate_deriv(R.f[k], L.invTd, r.f[k], sg);
        }
    }
}
__device__ __forceinline__ void rates_serial_f(const TLevel &L, int case_b, unsigned needF, unsigned needD, Rates &r)
{
    const RateFnTab &R = c_rate_fn[case_b];
#pragma unroll
    for (int k = 0; k < NRF; ++k) {
        if (needF & rf_bit(k)) {
            double df;
            rate_value_f(R.f[k], L, r.f[k], df);
            if (needD & rf_bit(k)) r.df[k] = df;
        }
    }
}

// a full warp (all 32 lanes, the same T): lane k's function k
template <bool MIX>
__device__ __forceinline__ void rate_lane(const TLevel &L, int case_b, double &f, double &df)
{
    const RateFn &q = g_rate_fn[case_b].f[threadIdx.x & 31];
    if constexpr (MIX) {
        rate_value_f(q, L, f, df);
    } else {
        using namespace dfm;
        double sg;
        const F2 l = rate_softplus(q, L, sg);
        const F2 arg = add(add(add(q.c0, mul(L.lnT, q.c1)), mul(L.invT, q.c2)), neg(mul(l, q.c3)));
        f = rmul(q.Cc, exp2d_inl(arg));
        df = rate_deriv(q, L.invTd, f, sg);
    }
}
// ... and the needed ones in every lane
template <bool MIX>
__device__ __forceinline__ void rates_warp(const TLevel &L, int case_b, unsigned needF, unsigned needD, Rates &r)
{
    double f, df;
    rate_lane<MIX>(L, case_b, f, df);
#pragma unroll
    for (int k = 0; k < NRF; ++k) {
        if (needF & rf_bit(k)) r.f[k] = __shfl_sync(0xffffffffu, f, k);
        if (needD & rf_bit(k)) r.df[k] = __shfl_sync(0xffffffffu, df, k);
    }
}

// A dual temperature (level L of its value, derivative dT): values as in
// rates_serial (the bits of the double path); with g = c1 - c2/T - c3 c4
// sigma, d ln f/dT = g/T and
//     d2f/dT2 = f [(g/T)^2 + (-g + c2/T - c3 c4^2 sigma (1 - sigma)) / T^2],
// so f carries df dT and df carries d2f dT.
__device__ __forceinline__ void rates_dual(const TLevel &L, double dT, int case_b, unsigned needF, unsigned needD,
                                           RatesT<Dual> &r)
{
    const RateFnTab &R = c_rate_fn[case_b];
    const double x = L.invTd;
#pragma unroll
    for (int k = 0; k < NRF; ++k) {
        if (needF & rf_bit(k)) {
            const RateFn &q = R.f[k];
            double sg;
            const double f = rate_value(q, L, sg);
            const double df = rate_deriv(q, x, f, sg);
            r.f[k] = Dual(f, df * dT);
            if (needD & rf_bit(k)) {
                const double g = q.d1 - q.d2 * x - q.d34 * sg;
                const double D = g * x;
                const double d2f = f * (D * D + x * x * (-g + q.d2 * x - q.d344 * sg * (1.0 - sg)));
                r.df[k] = Dual(df, d2f * dT);
            }
        }
    }
}

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

template <typename S>
__device__ __forceinline__ void h_rates_from(const RatesT<S> &t, HRatesT<S> &r)
{
    r.beta = t.f[RF_BETA_HI];
    r.dbeta = t.df[RF_BETA_HI];
    r.alpha = t.f[RF_ALPHA_HII];
    r.dalpha = t.df[RF_ALPHA_HII];
}

template <typename S>
__device__ __forceinline__ void he_rates_from(const RatesT<S> &t, HeRatesT<S> &r)
{
    r.beta_HeI = t.f[RF_BETA_HEI];
    r.beta_HeII = t.f[RF_BETA_HEII];
    r.alpha_HeII = t.f[RF_ALPHA_HEII];
    r.alpha_HeIII = t.f[RF_ALPHA_HEIII];
}

// Recombination rates of HII, HeII, HeIII (the case t was evaluated with)
template <typename S>
__device__ __forceinline__ void recomb_alphas(const RatesT<S> &t, S a[3])
{
    a[0] = t.f[RF_ALPHA_HII];
    a[1] = t.f[RF_ALPHA_HEII];
    a[2] = t.f[RF_ALPHA_HEIII];
}

// Primordial cooling magnitude L (Eq. (rate_cooling), positive = cooling)
// and dL/dT: the sum of the cooling functions (collisional ionisation and
// excitation, recombination and dielectronic cooling, bremsstrahlung) each
// times its density, in a fixed pairwise order, then Compton cooling.  All
// products and sums are rounded as written (rmul, radd), so the one-thread
// sum and the warp sum (lane k term k) give the same bits.
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
__device__ __forceinline__ void cooling_from(const RatesT<S> &t, double comp, double tg, bool helium, const S &T,
                                             const S &ne, const S &nHI, const S &nHII, const S &nHeI,
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
        if (helium || !q.he) {
            a[k] = rmul(t.f[RF_COOL0 + k], n[q.sp]);
            b[k] = rmul(t.df[RF_COOL0 + k], n[q.sp]);
        }
    }
    const S Ls = tree_sum16(a), dLs = tree_sum16(b);
    cooling_close(comp, tg, T, ne, Ls, dLs, L, dL);
}

// a full warp (all 32 lanes, the same arguments): lane k < 16 holds term k,
// the sums run over shuffles in the same pairwise order
template <bool MIX>
__device__ __forceinline__ void cooling_warp(int case_b, double comp, double tg, bool helium, double T, double ne,
                                             double nHI, double nHII, double nHeI, double nHeII, double nHeIII,
                                             double &L, double &dL)
{
    TLevel Lv;
    t_level<MIX, true>(T, Lv);
    double f, df;
    rate_lane<MIX>(Lv, case_b, f, df);
    double n[NSP];
    cool_densities(nHI, nHII, nHeI, nHeII, nHeIII, n);
    const int k = threadIdx.x & 15;
    const double nk = pick(n, g_cool_sp[k]);
    double v = rmul(f, nk), dv = rmul(df, nk);
    if (!helium && (cool_mask(1) & rf_bit(k))) v = dv = 0.0;
#pragma unroll
    for (int m = 8; m >= 1; m >>= 1) {
        v = radd(v, __shfl_xor_sync(0xffffffffu, v, m));
        dv = radd(dv, __shfl_xor_sync(0xffffffffu, dv, m));
    }
    // lanes 16..31 summed other functions: every lane takes lane 0's sums
    v = __shfl_sync(0xffffffffu, v, 0);
    dv = __shfl_sync(0xffffffffu, dv, 0);
    cooling_close(comp, tg, T, ne, v, dv, L, dL);
}

}  // namespace rtgb

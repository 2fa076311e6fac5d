// One thermo_step of the per-cell thermochemistry (paper App. A) and one
// attempt of its sub-cycling loop (Sec. 3.3.1), shared by the forward
// kernels (thermo.cu) and the adjoint's differentiated recomputation
// (adjoint.cu).  The scalar type S is double, or Dual for the adjoint.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "dual.cuh"
#include "rates.cuh"
#include "rt_internal.h"

namespace rtgb {
namespace thermo_detail {

constexpr double kEV = 1.602176634e-12;
constexpr double kEps0 = 13.60 * kEV, kEps1 = 24.59 * kEV, kEps2 = 54.42 * kEV;
constexpr double kFloorN = 1e-30;
constexpr double kXMin = 1e-6;
constexpr double kNeFloor = 1e-6;
constexpr double kTFloor = 1.0;

template <int G, typename S = double>
struct CellState {
    S x, y2, y3, T;
    S N[G];
    S Fs[G];          // accumulated flux scale prod 1/(1 + h D_i)
    S Nd[G];          // smoothed RT: photon density rate Ndot_i (Sec. 3.4)
    S Fb[G];          // smoothed RT: weight of Fdot_i in F, sum h prod 1/(1 + h D_i)
};

template <typename S = double>
struct IsoRates {     // quantities of a cell fixed over its sub-steps
    HRatesT<S> h;     // rates at the fixed temperature of an isothermal cell
    HeRatesT<S> he;
    S nHe, K, nef;    // n_He, (gamma - 1) X / (k_B n_H), the n_e floor 1e-6 n_H
};

template <typename S = double>
struct CoolCache {    // quantities of the current state at t, kept over rejected attempts
    S L, dL;          // cooling and dL/dT
    S rj[3];          // without the OTSA: (alpha^A_j - alpha^B_j) n_j n_e, j = HII, HeII, HeIII
    bool valid, rvalid;
};

template <typename S>
__device__ __forceinline__ void cell_constants(const ThermoParams &p, const S &nH, IsoRates<S> &iso)
{
    iso.nHe = nH * p.he_ratio;
    iso.K = p.kfac / nH;
    iso.nef = kNeFloor * nH;
}

// 1/mu, mu the mean particle mass in m_H (App. A)
template <typename S>
__device__ __forceinline__ S mu_den(double X, const S &x, const S &y2, const S &y3)
{
    return X * (1.0 + x) + 0.25 * (1.0 - X) * (1.0 + y2 + 2.0 * y3);
}

template <typename S>
__device__ __forceinline__ S mu_of(double X, const S &x, const S &y2, const S &y3)
{
    return qdiv(S(1.0), mu_den(X, x, y2, y3));
}


// Comparisons, minima and maxima of doubles through their bit patterns, on
// the integer pipe (a GB300 warp issues one FP64 instruction, compares and
// min/max included, per ~64 cycles).  For doubles >= +0 the signed 64-bit
// order of the bits is the order of the values, and every negative double
// orders below them, so these are exact wherever at most one operand can be
// negative; a NaN orders above +infinity.
constexpr long long kInfBits = 0x7ff0000000000000LL;

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// max(x, c), min(x, c) for c >= +0 and any x (dual numbers: fmax, fmin)
template <typename S, typename C>
__device__ __forceinline__ S max0(const S &x, C c)
{
    if constexpr (std::is_same<S, double>::value && std::is_same<C, double>::value)
        return __longlong_as_double(max(dbits(x), dbits(c)));
    else
        return fmax(x, c);
}

template <typename S, typename C>
__device__ __forceinline__ S min0(const S &x, C c)
{
    if constexpr (std::is_same<S, double>::value && std::is_same<C, double>::value)
        return __longlong_as_double(min(dbits(x), dbits(c)));
    else
        return fmin(x, c);
}

// 2 h and h / 2 of a positive normal h: the exponent moved by one (exact)
__device__ __forceinline__ double twice(double h)
{
    return (dbits(h) >> 52) < 2046 ? __longlong_as_double(dbits(h) + (1LL << 52)) : 2.0 * h;
}

__device__ __forceinline__ double half(double h)
{
    return (dbits(h) >> 52) > 1 ? __longlong_as_double(dbits(h) - (1LL << 52)) : 0.5 * h;
}

// fl(a / b) > t and fl(a / b) < t (a >= 0, b > 0), decided exactly as the
// rounded quotient would decide them: the product t b settles everything
// more than 8 ulps away from it (for doubles, by their bits; the rounding
// of t b and of the quotient is within 2 ulps), and the quotient itself is
// formed only inside that band (or for a NaN, which then compares false as
// the quotient would).  The 10% rule's decisions thus match a statement of
// it that divides, including at exact ties (a sub-cycled cell whose photon
// density grows linearly from zero meets relative changes of exactly 1/10
// and 1/20).  The quotient is kept out of line so that the compiler does
// not evaluate it on the common path.
template <typename S>
__device__ __noinline__ bool quotient_gt(S a, S b, double t)
{
    return a / b > t;
}

template <typename S>
__device__ __noinline__ bool quotient_lt(S a, S b, double t)
{
    return a / b < t;
}

template <typename S>
__device__ __forceinline__ bool ratio_gt(const S &a, const S &b, double t)
{
    const S tb = t * b;
    if constexpr (std::is_same<S, double>::value) {
        const long long ai = dbits(a), ti = dbits(tb);
        if (ai > ti + 8 && ai <= kInfBits) return true;
        if (ai < ti - 8) return false;
    } else {
        if (a > tb * (1.0 + 1e-15)) return true;
        if (a < tb * (1.0 - 1e-15)) return false;
    }
    return quotient_gt<S>(a, b, t);
}

template <typename S>
__device__ __forceinline__ bool ratio_lt(const S &a, const S &b, double t)
{
    const S tb = t * b;
    if constexpr (std::is_same<S, double>::value) {
        const long long ai = dbits(a), ti = dbits(tb);
        if (ai < ti - 8) return true;
        if (ai > ti + 8 && ai <= kInfBits) return false;
    } else {
        if (a < tb * (1.0 - 1e-15)) return true;
        if (a > tb * (1.0 + 1e-15)) return false;
    }
    return quotient_lt<S>(a, b, t);
}

template <bool WARP, bool MIX>
__device__ __forceinline__ void get_rates(const Dual &T, int case_b, unsigned needF, unsigned needD,
                                          RatesT<Dual> &r)
{
    static_assert(!WARP && !MIX, "dual rates: one thread, FP64");
    TLevel L;
    t_level<false>(T.v, L);
    rates_dual(L, T.d, case_b, needF, needD, r);
}
template <bool WARP, bool MIX>
__device__ __forceinline__ void rates_at(const TLevel &L, int case_b, unsigned needF, unsigned needD, Rates &r)
{
    if constexpr (WARP) rates_warp<MIX>(L, case_b, needF, needD, r);
    else if constexpr (MIX) rates_serial_f(L, case_b, needF, needD, r);
    else rates_serial(L, case_b, needF, needD, r);
}
template <bool WARP, bool MIX>
__device__ __forceinline__ void get_rates(double T, int case_b, unsigned needF, unsigned needD, Rates &r)
{
    TLevel L;
    t_level<MIX, WARP>(T, L);
    rates_at<WARP, MIX>(L, case_b, needF, needD, r);
}
// Rates at T = (T/mu') mu_j given 1/mu_j = md and 1/(T/mu') = iT as a pair
// (the helium temperatures of step 4 enter their rates only through 1/T and
// ln T): 1/T = md iT in pair arithmetic, no FP64 quotient.  A dual T takes
// the levels of its value and the derivative of Tmu1 / md.
__device__ __forceinline__ dfm::F2 inv_pair(double x)
{
    if (!(x > 0.0) || !dfm::splittable(x)) return dfm::split_any(1.0 / x);
    return dfm::rcp2(dfm::split(x));
}
template <bool WARP, bool MIX>
__device__ __forceinline__ void rates_mu(const Dual &md, dfm::F2 iT, const Dual &Tmu1, int case_b, unsigned needF,
                                         unsigned needD, RatesT<Dual> &r)
{
    static_assert(!WARP && !MIX, "dual rates: one thread, FP64");
    TLevel L;
    t_level_inv<false>(dfm::mul(dfm::split_any(md.v), iT), L);
    rates_dual(L, (Tmu1 / md).d, case_b, needF, needD, r);
}
template <bool WARP, bool MIX>
__device__ __forceinline__ void rates_mu(double md, dfm::F2 iT, double, int case_b, unsigned needF,
                                         unsigned needD, Rates &r)
{
    TLevel L;
    t_level_inv<MIX, WARP>(dfm::mul(dfm::split_any(md), iT), L);
    rates_at<WARP, MIX>(L, case_b, needF, needD, r);
}

// (alpha^A_j - alpha^B_j) n_j n_e of HII, HeII, HeIII at temperature T
// (Eq. (cool_N_cr)); out of line: it only runs without the OTSA, and
// inlined its two rate tables would raise the register count of every
// kernel
template <bool WARP, bool MIX, typename S>
__device__ __noinline__ void recomb_rates(S T, S nHII, S nHeII, S nHeIII, S ne, S *rj)
{
    S aA[3], aB[3];
    {
        RatesT<S> t;
        get_rates<WARP, MIX>(T, 0, kNeedRec, 0u, t);
        recomb_alphas(t, aA);
    }
    {
        RatesT<S> t;
        get_rates<WARP, MIX>(T, 1, kNeedRec, 0u, t);
        recomb_alphas(t, aB);
    }
    rj[0] = (aA[0] - aB[0]) * nHII * ne;
    rj[1] = (aA[1] - aB[1]) * nHeII * ne;
    rj[2] = (aA[2] - aB[2]) * nHeIII * ne;
}

// Photon update of one group, Eq. (SIE photons): N_i' = (N_i + h C_i)/(1 + h D_i)
// (C_i = 0 under the OTSA; smoothed RT adds the rate Ndot_i), F_i scaled by
// 1/(1 + h D_i), D_i = c_r sum_j sigma^N_ij n_j with the backward absorber
// densities; with the group's 10% and 5% checks on N_i and its terms of the
// photo-ionisation rates sigma^N_ij c_r N_i' (t0..t2) and of the
// photoheating c_r N_i' sum_j n_j (egy_i sigma^E_ij - eps_j sigma^N_ij)
// (tq).  Products and sums are rounded as written.
template <typename S>
struct PhotonTerms {
    S Nn, Fs, Fb, t0, t1, t2, tq;
    bool ok, small;
};

template <bool MIX, bool SM, typename S>
__device__ __forceinline__ void photon_group(const ThermoParams &p, int i, const S &N, const S &Fs, const S &Nd,
                                             const S &Fb, const S &Crec, const S &nHI, const S &nHeI,
                                             const S &nHeII, double h, PhotonTerms<S> &o)
{
    S inv;
    if constexpr (MIX) {
        // absorption coefficient in FP32; the update itself in FP64, since
        // a cell may take thousands of sub-steps and FP32 roundings of N
        // would accumulate past the stated 1e-4 (doubles narrowed and the
        // float widened through integer operations, not FP64-pipe
        // conversions)
        const float Df = __fadd_rn(__fadd_rn(__fmul_rn(narrow(p.crs[i][0]), narrow(nHI)),
                                             __fmul_rn(narrow(p.crs[i][1]), narrow(nHeI))),
                                   __fmul_rn(narrow(p.crs[i][2]), narrow(nHeII)));
        inv = qdiv(1.0, rfma(h, dfm::widen(Df), 1.0));
    } else {
        const S D = rfma(p.crs[i][2], nHeII, rfma(p.crs[i][1], nHeI, rmul(nHI, p.crs[i][0])));
        inv = qdiv(S(1.0), rfma(h, D, S(1.0)));
    }
    // smoothed RT: N + h Ndot rounded step by step, so a cell growing
    // linearly from zero meets its relative changes 1/k exactly
    S Nn;
    if constexpr (SM) Nn = rmul(radd(N, rmul(Nd + Crec, h)), inv);
    else if (p.emit) Nn = rmul(rfma(h, Crec, N), inv);
    else Nn = rmul(N, inv);
    const S dN = fabs(radd(Nn, -N)), den = max0(N, kFloorN);
    o.ok = !ratio_gt(dN, den, 0.1);
    o.small = ratio_lt(dN, den, 0.05);
    o.Nn = Nn;
    o.Fs = rmul(Fs, inv);
    if constexpr (SM) o.Fb = rmul(radd(Fb, S(h)), inv);
    const S crN = rmul(Nn, p.cr);
    o.t0 = rmul(crN, p.gc.sigN[i][0]);
    o.t1 = rmul(crN, p.gc.sigN[i][1]);
    o.t2 = rmul(crN, p.gc.sigN[i][2]);
    o.tq = rmul(crN, rfma(p.hq[i][2], nHeII, rfma(p.hq[i][1], nHeI, rmul(nHI, p.hq[i][0]))));
}

// a double or a dual from lane `src` of the warp
__device__ __forceinline__ double shfl_s(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ Dual shfl_s(const Dual &v, int src)
{
    return Dual(__shfl_sync(0xffffffffu, v.v, src), __shfl_sync(0xffffffffu, v.d, src));
}

// The photon stage of an attempt (group i on lane i of a warp), filling the
// new N_i, flux scales, the photo-ionisation rates gam_j and the
// photoheating; false when a group breaks the 10% rule.  The recombination
// photons C_i (without the OTSA) come from cc.rj.
template <int G, bool MIX, bool SM, typename S>
__device__ __forceinline__ bool photons_warp(const ThermoParams &p, const CellState<G, S> &s, const CoolCache<S> &cc,
                                             const S &nHI, const S &nHeI, const S &nHeII, double h,
                                             CellState<G, S> &o, S &gam0, S &gam1, S &gam2, S &heat, bool &sm)
{
    PhotonTerms<S> pt;
    const int lane = threadIdx.x & 31;
    const int gi = lane < G ? lane : 0;
    S Crec = 0.0;
    if (p.emit) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
            if (p.rec_g[j] == gi) Crec += cc.rj[j];
    }
    photon_group<MIX, SM>(p, gi, s.N[gi], s.Fs[gi], s.Nd[gi], s.Fb[gi], Crec, nHI, nHeI, nHeII, h, pt);
    const unsigned full = 0xffffffffu;
    const bool ok = !__any_sync(full, lane < G && !pt.ok);
    sm = sm && (__all_sync(full, lane >= G || pt.small) != 0);
#pragma unroll
    for (int i = 0; i < G; ++i) {
        o.N[i] = shfl_s(pt.Nn, i);
        o.Fs[i] = shfl_s(pt.Fs, i);
        if constexpr (SM) {
            o.Fb[i] = shfl_s(pt.Fb, i);
            o.Nd[i] = s.Nd[i];
        }
        const S t0 = shfl_s(pt.t0, i), t1 = shfl_s(pt.t1, i), t2 = shfl_s(pt.t2, i), tq = shfl_s(pt.tq, i);
        if (i == 0) {
            gam0 = t0; gam1 = t1; gam2 = t2; heat = tq;
        } else {
            gam0 = radd(gam0, t0); gam1 = radd(gam1, t1); gam2 = radd(gam2, t2); heat = radd(heat, tq);
        }
    }
    return ok;
}

template <int G, bool MIX, bool SM, typename S>
__device__ __forceinline__ bool photons_serial(const ThermoParams &p, const CellState<G, S> &s,
                                               const CoolCache<S> &cc, const S &nHI, const S &nHeI, const S &nHeII,
                                               double h, CellState<G, S> &o, S &gam0, S &gam1, S &gam2, S &heat,
                                               bool &sm)
{
    PhotonTerms<S> pt;
#pragma unroll
    for (int i = 0; i < G; ++i) {
        S Crec = 0.0;
        if (p.emit) {
#pragma unroll
            for (int j = 0; j < 3; ++j)
                if (p.rec_g[j] == i) Crec += cc.rj[j];
        }
        photon_group<MIX, SM>(p, i, s.N[i], s.Fs[i], s.Nd[i], s.Fb[i], Crec, nHI, nHeI, nHeII, h, pt);
        if (!pt.ok) return false;
        sm = sm && pt.small;
        o.N[i] = pt.Nn;
        o.Fs[i] = pt.Fs;
        if constexpr (SM) {
            o.Fb[i] = pt.Fb;
            o.Nd[i] = s.Nd[i];
        }
        if (i == 0) {
            gam0 = pt.t0; gam1 = pt.t1; gam2 = pt.t2; heat = pt.tq;
        } else {
            gam0 = radd(gam0, pt.t0); gam1 = radd(gam1, pt.t1); gam2 = radd(gam2, pt.t2);
            heat = radd(heat, pt.tq);
        }
    }
    return true;
}

// The two warps of a pair of the tail kernel (thermo_hard): while one evaluates
// the cooling at T(t) the other updates the photons; each posts its results
// in shared memory with a sequence number and waits (bounded) for the
// other's.  Both then hold the same values and run the rest of the attempt
// in step.  Two buffers alternate, so a post never overwrites data the
// partner may still be reading (every exchange is two-way).
template <int G>
struct PairX {
    double N[2][G], Fs[2][G], Fb[2][G], g[2][4], L[2], dL[2], m[2][3];
    int ok[2], small[2];
    unsigned long long item[2];
    volatile int seq[2];   // last exchange posted by role 0, role 1
};

struct PairCtx {
    void *x;          // PairX<G> of the pair, shared memory
    int role;         // 0: photons, 1: cooling
    int n;            // exchanges so far (the same in both warps)
    bool failed;      // a wait ran out (status set; the cell is abandoned)
};

constexpr long long kPairSpinLimit = 1LL << 24;   // polls before a wait gives up

// post this warp's part of exchange pc.n, then wait for the partner's
__device__ __forceinline__ void pair_post(volatile int *seq_mine, int n)
{
    __threadfence_block();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) *seq_mine = n;
}

__device__ __forceinline__ bool pair_wait(volatile int *seq_other, int n, unsigned *status)
{
    bool ok = true;
    if ((threadIdx.x & 31) == 0) {
        long long k = 0;
        while (*seq_other < n && k < kPairSpinLimit) {
            __nanosleep(32);
            ++k;
        }
        ok = *seq_other >= n;
        if (!ok) atomicOr(status, kStatusQueue);
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    __threadfence_block();
    return ok;
}

// One thermo_step over h.  Returns true and fills `o` when the 10% rule
// holds; `small` then tells whether every checked change stayed below 5%.
// The checks |dX| / den > 0.1 go through ratio_gt / ratio_lt (a division
// only near the threshold).
// MIX (RT_MIXED32): the rates' softplus corrections and exponentials and
// the absorption coefficients in FP32 (rates.cuh, rate_value_f); the
// photon, T/mu, x_HII and helium updates and 1 - x in FP64.
//
// S is double, or Dual for the adjoint's differentiated recomputation
// (values bit-identical to the double path; MIX only with double).
template <int G, bool WARP, bool MIX, typename S = double, bool SM = false, bool PAIR = false>
__device__ __forceinline__ bool attempt(const ThermoParams &p, const S &nH, const CellState<G, S> &s, double h,
                                        const IsoRates<S> &iso, CoolCache<S> &cc, CellState<G, S> &o,
                                        bool &small, PairCtx *pc = nullptr, unsigned *status = nullptr)
{
    static_assert(!PAIR || (WARP && sizeof(S) == sizeof(double)), "pairs of warps: the warp path");
    static_assert(!MIX || sizeof(S) == sizeof(double), "the mixed path is not differentiated");
    const S nHe = iso.nHe;
    const S x = s.x, y2 = s.y2, y3 = s.y3;
    const S nHI = nH * (1.0 - x);
    const S nHII = nH * x;
    const S nHeI = nHe * (1.0 - y2 - y3);
    const S nHeII = nHe * y2;
    const S nHeIII = nHe * y3;
    const S ne = nHII + (y2 + 2.0 * y3) * nHe;
    const double cr = p.cr;
    bool sm = true;
    S gam0 = 0.0, gam1 = 0.0, gam2 = 0.0, heat = 0.0;

    // cooling at T(t) and the state at t (step 2 below), first: it depends on
    // nothing this sub-step computes, so its rate functions can overlap the
    // photon update; kept over rejected attempts
    // recombination photons without the OTSA, Eq. (cool_N_cr), at T(t) with
    // the backward abundances; group i gains C_i = sum_j [rec_g[j] == i] rj[j]
    // (before the cooling: a pair of warps updates the photons there)
    if (p.emit && !cc.rvalid) {
        recomb_rates<WARP, MIX>(s.T, nHII, nHeII, nHeIII, ne, cc.rj);
        cc.rvalid = true;
    }

    bool pair_photons = false;   // the photon stage was done in the pair exchange
    // the parts of step 2 that depend on the state only: 1/mu, mu, T/mu
    S mden, mu, Tmu;
    bool have_mu = false;
    if (!p.isothermal && !cc.valid) {
        if constexpr (PAIR) {
            // role 1 evaluates the cooling, role 0 the photon stage, at once
            PairX<G> &X = *static_cast<PairX<G> *>(pc->x);
            const int b = pc->n & 1;
            const int n = ++pc->n;
            const int lane = threadIdx.x & 31;
            if (pc->role == 1) {
                cooling_warp<MIX>(p.case_b, p.comp, p.tg, p.helium != 0, s.T, ne, nHI, nHII, nHeI, nHeII, nHeIII,
                                  cc.L, cc.dL);
                if (lane == 0) {
                    X.L[b] = cc.L;
                    X.dL[b] = cc.dL;
                }
                pair_post(&X.seq[1], n);
                if (!pair_wait(&X.seq[0], n, status)) { pc->failed = true; return false; }
                if (!X.ok[b]) { cc.valid = true; return false; }
#pragma unroll
                for (int i = 0; i < G; ++i) {
                    o.N[i] = X.N[b][i];
                    o.Fs[i] = X.Fs[b][i];
                    if constexpr (SM) {
                        o.Fb[i] = X.Fb[b][i];
                        o.Nd[i] = s.Nd[i];
                    }
                }
                gam0 = X.g[b][0]; gam1 = X.g[b][1]; gam2 = X.g[b][2]; heat = X.g[b][3];
                sm = X.small[b] != 0;
                mden = X.m[b][0]; mu = X.m[b][1]; Tmu = X.m[b][2];
            } else {
                const bool ok = photons_warp<G, MIX, SM>(p, s, cc, nHI, nHeI, nHeII, h, o, gam0, gam1, gam2, heat, sm);
                // (this warp would wait for the cooling meanwhile)
                mden = mu_den(p.X, x, y2, y3);
                mu = qdiv(S(1.0), mden);
                Tmu = s.T * mden;
                if (lane == 0) {
                    X.m[b][0] = mden; X.m[b][1] = mu; X.m[b][2] = Tmu;
#pragma unroll
                    for (int i = 0; i < G; ++i) {
                        X.N[b][i] = o.N[i];
                        X.Fs[b][i] = o.Fs[i];
                        if constexpr (SM) X.Fb[b][i] = o.Fb[i];
                    }
                    X.g[b][0] = gam0; X.g[b][1] = gam1; X.g[b][2] = gam2; X.g[b][3] = heat;
                    X.ok[b] = ok;
                    X.small[b] = sm;
                }
                pair_post(&X.seq[0], n);
                if (!pair_wait(&X.seq[1], n, status)) { pc->failed = true; return false; }
                cc.L = X.L[b];
                cc.dL = X.dL[b];
                if (!ok) { cc.valid = true; return false; }
            }
            cc.valid = true;
            pair_photons = true;
            have_mu = true;
        } else {
            if constexpr (WARP) {   // lane k evaluates cooling term k
                cooling_warp<MIX>(p.case_b, p.comp, p.tg, p.helium != 0, s.T, ne, nHI, nHII, nHeI, nHeII, nHeIII,
                                  cc.L, cc.dL);
            } else {
                const unsigned need = kNeedCoolH | (p.helium ? kNeedCoolHe : 0u);
                RatesT<S> t;
                get_rates<WARP, MIX>(s.T, p.case_b, need, need, t);
                cooling_from(t, p.comp, p.tg, p.helium != 0, s.T, ne, nHI, nHII, nHeI, nHeII, nHeIII, cc.L, cc.dL);
            }
            cc.valid = true;
        }
    }


    // 1. photons: group i's update depends on no other group, so the warp
    // path gives group i to lane i; the one-thread path loops over the
    // groups; both call photon_group and sum the groups' terms in the same
    // order (rounded as written), so they give the same bits
    if (!pair_photons) {
        bool ok;
        if constexpr (WARP) ok = photons_warp<G, MIX, SM>(p, s, cc, nHI, nHeI, nHeII, h, o, gam0, gam1, gam2, heat, sm);
        else ok = photons_serial<G, MIX, SM>(p, s, cc, nHI, nHeI, nHeII, h, o, gam0, gam1, gam2, heat, sm);
        if (!ok) return false;
    }
    if (p.isothermal) heat = 0.0;

    // 2. temperature: T/mu + K h (Lambda) / (1 + mu (dL/dT) K h), Lambda =
    // heating - cooling, d Lambda/d(T/mu) = -mu dL/dT
    if (!have_mu) {
        mden = mu_den(p.X, x, y2, y3);
        mu = qdiv(S(1.0), mden);
        Tmu = s.T * mden;
    }
    S Tmu1 = 0.0;
    if (!p.isothermal) {
        const S Kh = iso.K * h;
        const S num = (heat - cc.L) * Kh;
        const S dT = qdiv(num, 1.0 + (mu * cc.dL) * Kh);
        Tmu1 = Tmu + dT;
        S adT = fabs(dT);
        if (ratio_gt(fabs(num), Tmu, 0.1)) return false;
        if (ratio_gt(adT, Tmu, 0.1)) return false;
        sm = sm && ratio_lt(adT, Tmu, 0.05);
    }
    // 1/(T/mu') as a pair, for the helium temperatures (T/mu') mu_j
    const dfm::F2 iT = (p.isothermal || !p.helium) ? dfm::F2{0.0f, 0.0f} : inv_pair(val(Tmu1));

    // 3. hydrogen
    HRatesT<S> hr;
    if (p.isothermal) {
        hr = iso.h;
    } else {
        RatesT<S> t;
        get_rates<WARP, MIX>(Tmu1 * mu, p.case_b, kNeedH, kNeedH, t);
        h_rates_from(t, hr);
    }
    S C = hr.beta * ne + gam0;
    S Dd = hr.alpha * ne;
    S dC = nH * hr.beta, dD = nH * hr.alpha;
    if (!p.isothermal) {
        S f = ne * Tmu1 * mu * mu * p.X;
        dC -= f * hr.dbeta;
        dD -= f * hr.dalpha;
    }
    S J = dC - (C + Dd) - x * (dC + dD);
    S xdot = C - x * (C + Dd);
    S x1 = x + qdiv(h * xdot, 1.0 - J * h);
    x1 = min0(max0(x1, kXMin), 1.0);
    {
        S xden = max0(x, kXMin);
        S dx = fabs(x1 - x);
        if (ratio_gt(dx, xden, 0.1)) return false;
        if (ratio_gt(fabs(xdot) * h, xden, 0.1)) return false;
        sm = sm && ratio_lt(dx, xden, 0.05);
    }

    // 4. helium
    S y2n = y2, y3n = y3;
    if (p.helium) {
        S yI = 1.0 - y2 - y3;
        S ne2 = x1 * nH + (y2 + 2.0 * y3) * nHe;
        HeRatesT<S> r2;
        if (p.isothermal) {
            r2 = iso.he;
        } else {
            RatesT<S> t;
            rates_mu<WARP, MIX>(mu_den(p.X, x1, y2, y3), iT, Tmu1, p.case_b, kNeedHe, 0u, t);
            he_rates_from(t, r2);
        }
        S C1 = y2 * r2.alpha_HeII * ne2;
        S D1 = r2.beta_HeI * ne2 + gam1;
        S yI1 = qdiv(yI + C1 * h, 1.0 + D1 * h);
        S C2 = yI1 * (r2.beta_HeI * ne2 + gam1) + y3 * r2.alpha_HeIII * ne2;
        S D2 = (r2.beta_HeII + r2.alpha_HeII) * ne2 + gam2;
        y2n = qdiv(y2 + C2 * h, 1.0 + D2 * h);
        S ne3 = x1 * nH + (y2n + 2.0 * y3) * nHe;
        HeRatesT<S> r3;
        if (p.isothermal) {
            r3 = iso.he;
        } else {
            RatesT<S> t;
            rates_mu<WARP, MIX>(mu_den(p.X, x1, y2n, y3), iT, Tmu1, p.case_b, kNeedHe3, 0u, t);
            r3.beta_HeII = t.f[RF_BETA_HEII];
            r3.alpha_HeIII = t.f[RF_ALPHA_HEIII];
        }
        S C3 = y2n * (r3.beta_HeII * ne3 + gam2);
        S D3 = r3.alpha_HeIII * ne3;
        y3n = qdiv(y3 + C3 * h, 1.0 + D3 * h);
        // conservation: lower the largest fraction (HeI largest: no change)
        if (y2n >= yI1 && y2n >= y3n) y2n = 1.0 - yI1 - y3n;
        else if (y3n >= yI1 && y3n > y2n) y3n = 1.0 - yI1 - y2n;
        y2n = min0(max0(y2n, 0.0), 1.0);
        y3n = min0(max0(y3n, 0.0), 1.0);
    }
    {
        S ne1 = x1 * nH + (y2n + 2.0 * y3n) * nHe;
        S dne = fabs(ne1 - ne), den = max0(ne, iso.nef);
        if (ratio_gt(dne, den, 0.1)) return false;
        sm = sm && ratio_lt(dne, den, 0.05);
    }
    S Tf = p.isothermal ? s.T : qdiv(Tmu1, mu_den(p.X, x1, y2n, y3n));
    o.x = x1;
    o.y2 = y2n;
    o.y3 = y3n;
    o.T = max0(Tf, kTFloor);
    small = sm;
    return true;
}

// One attempt of the sub-cycling loop; returns true when the cell is done.
template <int G, bool WARP, bool MIX, typename S = double, bool SM = false, bool PAIR = false>
__device__ __forceinline__ bool subcycle_once(const ThermoParams &p, const S &nH, CellState<G, S> &st,
                                              double &t_left, double &dt_tc, int &att, const IsoRates<S> &iso,
                                              CoolCache<S> &cc, PairCtx *pc = nullptr, unsigned *status = nullptr)
{
    // t_left, dt_tc > 0: compared through their bits
    double h = (dbits(dt_tc) < dbits(t_left)) ? dt_tc : t_left;
    ++att;
    CellState<G, S> o;
    bool small = false;
    if (attempt<G, WARP, MIX, S, SM, PAIR>(p, nH, st, h, iso, cc, o, small, pc, status)) {
        st = o;
        cc.valid = false;
        cc.rvalid = false;
        t_left = (dbits(h) == dbits(t_left)) ? 0.0 : t_left - h;
        dt_tc = small ? twice(h) : h;
    } else {
        dt_tc = half(h);
    }
    return dbits(t_left) <= 0;
}

}  // namespace thermo_detail
}  // namespace rtgb

// Thermochemistry kernels (first pass, lane-per-cell drains, pair-of-warps
// tail) and their launch sequence, templated on the group count G, the
// photon storage type P (double: RT_FP64; float: RT_MIXED), FP32 rate
// transcendentals R32 (RT_MIXED32) and smoothed RT SM (Sec. 3.4).  Each
// launcher translation unit instantiates one (P, R32) family, so the
// families compile in parallel.
//
// Smoothed RT: on entry N, F hold the result N', F' of injection and
// transport and Npre, Fpre the state before them.  The first pass loads
// N^t = Npre and Ndot = (N' - N^t)/dt per group; a cell's flux is kept as
// F = Fs F_base + Fb Fdot with Fs = prod 1/(1 + h D), Fb = sum h prod
// 1/(1 + h D) over its accepted sub-steps.  A cell handed to a queue
// leaves its partial N, F in N, F and its Ndot, Fdot in Npre, Fpre.
#pragma once

#include <cuda_runtime.h>

#include "rates.cuh"
#include "rt_internal.h"
#include "thermo_step.cuh"

namespace rtgb {
namespace {

using namespace thermo_detail;

constexpr int kPass1Block = 128;

// first: the cell's first load in this RT step (thermo_pass1)
template <int G, bool WARP, typename P, bool R32, bool SM>
__device__ __forceinline__ void load_cell(const ThermoParams &p, long long c, bool first, const double *xHII,
                                          const double *xHeII, const double *xHeIII, const double *T,
                                          const P *N, const P *Npre, const double *fscale, CellState<G> &st,
                                          IsoRates<> &iso, CoolCache<> &cc)
{
    st.x = xHII[c];
    st.y2 = xHeII[c];
    st.y3 = xHeIII[c];
    st.T = T[c];
#pragma unroll
    for (int i = 0; i < G; ++i) {
        const long long k = (long long)i * p.nc + c;
        if constexpr (SM) {
            if (first) {
                const double n0 = (double)Npre[k];
                st.Nd[i] = ((double)N[k] - n0) / p.dt;   // Eq. (smoothrate1)
                st.N[i] = n0;
            } else {
                st.N[i] = (double)N[k];
                st.Nd[i] = (double)Npre[k];
            }
            st.Fb[i] = first ? 0.0 : fscale[(long long)(G + i) * p.nc + c];
        } else {
            st.N[i] = (double)N[k];
        }
        st.Fs[i] = first ? 1.0 : fscale[k];
    }
    cc.valid = false;
    cc.rvalid = false;
    if (p.isothermal) {
        Rates t;
        get_rates<WARP, R32>(st.T, p.case_b, kNeedH | (p.helium ? kNeedHe : 0u), kNeedH, t);
        h_rates_from(t, iso.h);
        if (p.helium) he_rates_from(t, iso.he);
    }
}

// handoff: the cell goes to a queue unfinished.  Its flux scale (and Fdot
// weight) then goes to fscale and F keeps F_base: the flux is formed once,
// when the cell finishes, so it does not depend on where it sub-cycled.
template <int G, typename P, bool SM>
__device__ __forceinline__ void store_cell(const ThermoParams &p, long long c, bool first, bool handoff,
                                           double *xHII, double *xHeII, double *xHeIII, double *T, P *N, P *F,
                                           P *Npre, P *Fpre, double *fscale, const CellState<G> &st,
                                           unsigned *status)
{
    xHII[c] = st.x;
    xHeII[c] = st.y2;
    xHeIII[c] = st.y3;
    T[c] = st.T;
    bool bad = !isfinite(st.x) || !isfinite(st.T);
#pragma unroll
    for (int i = 0; i < G; ++i) {
        N[(long long)i * p.nc + c] = (P)st.N[i];
        bad |= !isfinite(st.N[i]);
        if (handoff) {
            fscale[(long long)i * p.nc + c] = st.Fs[i];
            if constexpr (SM) fscale[(long long)(G + i) * p.nc + c] = st.Fb[i];
        }
        if constexpr (SM) {
            if (handoff && !first) continue;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const long long b = (3LL * i + d) * p.nc + c;
                double base, fd;
                if (first) {
                    base = (double)Fpre[b];
                    fd = ((double)F[b] - base) / p.dt;   // Eq. (smoothrate2)
                } else {
                    base = (double)F[b];
                    fd = (double)Fpre[b];
                }
                if (handoff) {
                    F[b] = Fpre[b];
                    Fpre[b] = (P)fd;
                } else {
                    F[b] = (P)(st.Fs[i] * base + st.Fb[i] * fd);
                }
            }
            if (handoff) Npre[(long long)i * p.nc + c] = (P)st.Nd[i];
        } else if (!handoff && st.Fs[i] != 1.0) {
            long long b = 3LL * i * p.nc + c;
            const P f = (P)st.Fs[i];
            F[b] *= f;
            F[b + p.nc] *= f;
            F[b + 2 * p.nc] *= f;
        }
    }
    if (bad) atomicOr(status, kStatusNonFinite);
}

__device__ __forceinline__ void push_item(const QueueArrays &a, unsigned long long slot, long long cap, uint32_t c,
                                          double t_left, double dt_tc, int att, unsigned *status)
{
    if (slot < (unsigned long long)cap) {
        a.cell[slot] = c;
        a.t_left[slot] = t_left;
        a.dt_tc[slot] = dt_tc;
        a.attempts[slot] = att;
    } else {
        atomicOr(status, kStatusQueue);
    }
}

template <int G, typename P, bool R32, bool SM>
__global__ void __launch_bounds__(kPass1Block)
thermo_pass1(ThermoParams p, const double *__restrict__ nH, double *xHII, double *xHeII, double *xHeIII,
             double *T, P *N, P *F, P *Npre, P *Fpre, int32_t *subcycles, Queue q, unsigned *status)
{
    long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = c < p.nc;
    bool push = false;
    double t_left = p.dt, dt_tc = p.dt;
    int att = 0;
    if (valid) {
        CellState<G> st;
        IsoRates<> iso;
        CoolCache<> cc;
        load_cell<G, false, P, R32, SM>(p, c, true, xHII, xHeII, xHeIII, T, N, Npre, q.fscale, st, iso, cc);
        double n = nH[c];
        cell_constants(p, n, iso);
        bool done = false;
        const int lim = p.pass1_attempts < p.max_sub ? p.pass1_attempts : p.max_sub;
        for (int k = 0; k < lim && !done; ++k)
            done = subcycle_once<G, false, R32, double, SM>(p, n, st, t_left, dt_tc, att, iso, cc);
        if (!done && att >= p.max_sub) {
            atomicOr(status, kStatusSubcycle);
            done = true;
        }
        store_cell<G, P, SM>(p, c, true, !done, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, q.fscale, st, status);
        if (done) subcycles[c] = att;
        else push = true;
    }
    // warp-aggregated append of unfinished cells to queue A
    unsigned m = __ballot_sync(0xffffffffu, push);
    if (m) {
        int lane = threadIdx.x & 31;
        int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(&q.counters[0], (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (push)
            push_item(q.a, base + __popc(m & ((1u << lane) - 1u)), q.capacity, (uint32_t)c, t_left, dt_tc, att,
                      status);
    }
}

// One lane-per-cell drain stage: cells of queue `src` (count and head in
// counters[cnt], counters[cnt + 1]) sub-cycle here for at most `budget`
// attempts; a cell still unfinished moves to queue `dst` (count in
// counters[dst_cnt]).  When `src` holds no more than `pass_below` cells the
// stage only moves them to `dst`: so few long sub-cyclers finish sooner one
// warp each than sharing warps.
struct DrainStage {
    QueueArrays src, dst;
    int cnt, dst_cnt, budget;
    long long pass_below;
};

template <int G, typename P, bool R32, bool SM>
__global__ void __launch_bounds__(128)
thermo_drain(ThermoParams p, const double *__restrict__ nH, double *xHII, double *xHeII, double *xHeIII,
             double *T, P *N, P *F, P *Npre, P *Fpre, int32_t *subcycles, Queue q, DrainStage ds,
             unsigned *status)
{
    unsigned long long count = q.counters[ds.cnt];
    if (count > (unsigned long long)q.capacity) count = (unsigned long long)q.capacity;
    if (count == 0) return;
    if ((long long)count <= ds.pass_below) {
        const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        for (long long it = gt; it < (long long)count; it += (long long)gridDim.x * blockDim.x) {
            ds.dst.cell[it] = ds.src.cell[it];
            ds.dst.t_left[it] = ds.src.t_left[it];
            ds.dst.dt_tc[it] = ds.src.dt_tc[it];
            ds.dst.attempts[it] = ds.src.attempts[it];
        }
        if (gt == 0) q.counters[ds.dst_cnt] = count;
        return;
    }
    CellState<G> st;
    IsoRates<> iso;
    CoolCache<> cc;
    double t_left = 0.0, dt_tc = 0.0, n = 0.0;
    int att = 0, used = 0;
    long long c = -1;
    bool have = false;
    auto fetch = [&]() {
        unsigned long long it = atomicAdd(&q.counters[ds.cnt + 1], 1ULL);
        if (it < count) {
            c = ds.src.cell[it];
            t_left = ds.src.t_left[it];
            dt_tc = ds.src.dt_tc[it];
            att = ds.src.attempts[it];
            n = nH[c];
            used = 0;
            load_cell<G, false, P, R32, SM>(p, c, false, xHII, xHeII, xHeIII, T, N, Npre, q.fscale, st, iso, cc);
            cell_constants(p, n, iso);
            have = true;
        } else {
            have = false;
        }
    };
    fetch();
    while (have) {
        bool done = subcycle_once<G, false, R32, double, SM>(p, n, st, t_left, dt_tc, att, iso, cc);
        if (!done && att >= p.max_sub) {
            atomicOr(status, kStatusSubcycle);
            done = true;
        }
        if (done) {
            store_cell<G, P, SM>(p, c, false, false, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, q.fscale, st, status);
            subcycles[c] = att;
            fetch();
        } else if (++used >= ds.budget) {
            // long sub-cycler: hand it to the next stage
            store_cell<G, P, SM>(p, c, false, true, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, q.fscale, st, status);
            unsigned long long slot = atomicAdd(&q.counters[ds.dst_cnt], 1ULL);
            push_item(ds.dst, slot, q.capacity, (uint32_t)c, t_left, dt_tc, att, status);
            fetch();
        }
    }
}

// The tail: a pair of warps per queued cell (warps 2k, 2k + 1 of a block).
// Both warps run the cell's attempts in step with identical state; in each
// attempt that needs the cooling at T(t), warp 2k + 1 evaluates it while
// warp 2k updates the photons (PairX exchange, thermo_step.cuh).  Warp 2k
// takes the next queue item and posts it to its partner the same way.  A
// wait that runs out (it cannot while both warps run the same code) sets
// the queue status bit and ends the pair.
template <int G, typename P, bool R32, bool SM>
__global__ void __launch_bounds__(128)
thermo_hard(ThermoParams p, const double *__restrict__ nH, double *xHII, double *xHeII, double *xHeIII,
            double *T, P *N, P *F, P *Npre, P *Fpre, int32_t *subcycles, Queue q, unsigned *status)
{
    unsigned long long count = q.counters[4];
    if (count > (unsigned long long)q.capacity) count = (unsigned long long)q.capacity;
    if (count == 0) return;
    __shared__ PairX<G> px[2];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int team = warp >> 1;
    PairCtx pc{&px[team], warp & 1, 0, false};
    if (lane == 0) px[team].seq[pc.role] = 0;
    __syncthreads();
    PairX<G> &X = px[team];
    while (true) {
        // the item: taken by role 0, posted to role 1 (exchange pc.n)
        const int b = pc.n & 1;
        const int n = ++pc.n;
        unsigned long long it = 0;
        if (pc.role == 0) {
            if (lane == 0) {
                it = atomicAdd(&q.counters[5], 1ULL);
                X.item[b] = it;
            }
            it = __shfl_sync(0xffffffffu, it, 0);
            pair_post(&X.seq[0], n);
            if (!pair_wait(&X.seq[1], n, status)) return;
        } else {
            pair_post(&X.seq[1], n);
            if (!pair_wait(&X.seq[0], n, status)) return;
            it = X.item[b];
        }
        if (it >= count) break;
        const long long c = q.a.cell[it];
        double t_left = q.a.t_left[it];
        double dt_tc = q.a.dt_tc[it];
        int att = q.a.attempts[it];
        const double n_h = nH[c];
        CellState<G> st;
        IsoRates<> iso;
        CoolCache<> cc;
        load_cell<G, true, P, R32, SM>(p, c, false, xHII, xHeII, xHeIII, T, N, Npre, q.fscale, st, iso, cc);
        cell_constants(p, n_h, iso);
        bool done = false;
        while (!done) {
            done = subcycle_once<G, true, R32, double, SM, true>(p, n_h, st, t_left, dt_tc, att, iso, cc, &pc, status);
            if (pc.failed) return;
            if (!done && att >= p.max_sub) {
                if (lane == 0 && pc.role == 0) atomicOr(status, kStatusSubcycle);
                done = true;
            }
        }
        if (lane == 0 && pc.role == 0) {
            store_cell<G, P, SM>(p, c, false, false, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, q.fscale, st, status);
            subcycles[c] = att;
        }
        __syncwarp();
    }
}

template <int G, typename P, bool R32, bool SM>
cudaError_t launch_g(const ThermoParams &tp, const double *nH, double *xHII, double *xHeII, double *xHeIII,
                     double *T, P *N, P *F, P *Npre, P *Fpre, int32_t *sub, Queue q, unsigned *status, int n_sm,
                     cudaStream_t s, cudaEvent_t *ev)
{
    const int B = kPass1Block;
    long long nb = (tp.nc + B - 1) / B;
    if (ev) cudaEventRecord(ev[0], s);
    thermo_pass1<G, P, R32, SM><<<(unsigned)nb, B, 0, s>>>(tp, nH, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, sub, q,
                                                          status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, thermo_drain<G, P, R32, SM>, 128, 0);
        if (per_sm < 1) per_sm = 1;
    }
    long long grid = (long long)per_sm * n_sm;
    long long need = (tp.nc + 127) / 128;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    // a pair of warps per long sub-cycler: two 4-warp blocks per SM
    long long hgrid = 2LL * n_sm;
    long long hneed = (tp.nc + 3) / 4;
    if (hgrid > hneed) hgrid = hneed;
    if (hgrid < 1) hgrid = 1;
    if (ev) { cudaEventRecord(ev[1], s); cudaEventRecord(ev[2], s); }
    DrainStage d1{q.a, q.b, 0, 2, tp.drain_budget, 0};
    thermo_drain<G, P, R32, SM><<<(unsigned)grid, 128, 0, s>>>(tp, nH, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, sub,
                                                              q, d1, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // many more long sub-cyclers than the tail kernel has pairs: they share
    // the FP64 pipes anyway, so a lane per cell does more per cycle; up to
    // eight cells per tail block (four per pair), the pairs keep each
    // cell's path short
    DrainStage d2{q.b, q.a, 2, 4, tp.drain2_budget, tp.drain2_min < 0 ? 8 * hgrid : tp.drain2_min};
    thermo_drain<G, P, R32, SM><<<(unsigned)grid, 128, 0, s>>>(tp, nH, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, sub,
                                                              q, d2, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    thermo_hard<G, P, R32, SM><<<(unsigned)hgrid, 128, 0, s>>>(tp, nH, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, sub, q,
                                                             status);
    if (ev) cudaEventRecord(ev[3], s);
    return cudaGetLastError();
}

template <typename P, bool R32, bool SM>
cudaError_t dispatch_g(const ThermoParams &tp, int G, const double *nH, double *xHII, double *xHeII, double *xHeIII,
                       double *T, P *N, P *F, P *Npre, P *Fpre, int32_t *sub, Queue q, unsigned *status, int n_sm,
                       cudaStream_t s, cudaEvent_t *ev)
{
#define RTGB_G(GG)                                                                                                 \
    case GG:                                                                                                       \
        return launch_g<GG, P, R32, SM>(tp, nH, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, sub, q, status, n_sm, s, \
                                        ev);
    switch (G) {
        RTGB_G(1)
        RTGB_G(2)
        RTGB_G(3)
        RTGB_G(4)
        RTGB_G(5)
        RTGB_G(6)
        RTGB_G(7)
        RTGB_G(8)
    default: return cudaErrorInvalidValue;
    }
#undef RTGB_G
}

}  // namespace
}  // namespace rtgb

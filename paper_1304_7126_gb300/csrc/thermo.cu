// Per-cell non-equilibrium thermochemistry (paper Sec. 3.3 and App. A),
// sub-cycled under the 10% rule (Sec. 3.3.1, App. A task 5), FP64.
//
// One thermo_step(h) follows App. A in its order, forward-in-time values
// wherever already updated, backward otherwise:
//   1. N_i, F_i semi-implicitly, Eq. (SIE photons) (OTSA: no creation term)
//   2. T/mu, Eq. (T integration num eq 2), heating Eq. (PHeat2) with the
//      new N_i, cooling Eq. (rate_cooling) at T(t) (skipped when isothermal)
//   3. x_HII, Eq. (xhii_update_2), rates at T = (T/mu)' mu(x(t))
//   4. x_HeI, x_HeII, x_HeIII, Eqs. (xhei_update), (xheii_update),
//      (xheiii_update), n_e and mu refreshed before each, then the helium
//      fractions renormalised by lowering the largest one
// and rejects the sub-step (halving it) when N_i, T/mu, x_HII or n_e move by
// more than 10%, or the first-order T and x_HII terms exceed 10%; after a
// sub-step whose largest change is below 5% the next one is doubled.  The
// cooling rate and its derivative depend only on the state at t, so a
// rejected sub-step keeps them for the retry.
//
// Load balance, three kernels per RT step:
//   thermo_pass1  one thread per cell (coalesced), up to 6 attempts; cells
//                 still sub-cycling go to queue A with their partial state;
//   thermo_drain  persistent; every lane takes queue-A items one at a time,
//                 one attempt per loop iteration, and fetches the next item
//                 as soon as its cell completes; a cell that needs more than
//                 kDrainBudget attempts here moves to queue B;
//   thermo_hard   persistent; one warp per queue-B cell.  On GB300 a lone
//                 FP64 dependent chain is slow (64 cycles per FMA, ~1000 per
//                 exp), so the lanes of the warp evaluate the cell's
//                 twenty-odd transcendentals of each temperature in parallel
//                 (rates.cuh, transc_warp) while the scalar update runs
//                 redundantly in all lanes.  The arithmetic is identical to
//                 the one-thread path, so results do not depend on which
//                 kernel finished a cell.
// Nothing waits on another thread; each kernel ends when its queue is empty.
#include <cuda_runtime.h>

#include <mutex>

#include "rates.cuh"
#include "rt_internal.h"
#include "thermo_step.cuh"

namespace rtgb {


namespace {

using namespace thermo_detail;

constexpr int kPass1Block = 128;
constexpr int kDrainBudget = 192;   // attempts a cell may spend in the first drain stage
constexpr int kDrain2Budget = 512;  // ... and in the second

template <int G, bool WARP, typename P, bool R32>
__device__ __forceinline__ void load_cell(const ThermoParams &p, long long c, const double *xHII,
                                          const double *xHeII, const double *xHeIII, const double *T,
                                          const P *N, CellState<G> &st, IsoRates<> &iso, CoolCache<> &cc)
{
    st.x = xHII[c];
    st.y2 = xHeII[c];
    st.y3 = xHeIII[c];
    st.T = T[c];
#pragma unroll
    for (int i = 0; i < G; ++i) {
        st.N[i] = (double)N[(long long)i * p.nc + c];
        st.Fs[i] = 1.0;
    }
    cc.valid = false;
    if (p.isothermal) {
        Transc t;
        get_transc<WARP, R32>(st.T, p.case_b, kNeedH | (p.helium ? kNeedHe : 0u), t);
        h_rates_from(t, p.case_b, iso.h);
        if (p.helium) he_rates_from(t, p.case_b, iso.he);
    }
}

template <int G, typename P>
__device__ __forceinline__ void store_cell(const ThermoParams &p, long long c, double *xHII, double *xHeII,
                                           double *xHeIII, double *T, P *N, P *F, const CellState<G> &st,
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
        if (st.Fs[i] != 1.0) {
            long long b = 3LL * i * p.nc + c;
            const P f = (P)st.Fs[i];
            F[b] *= f;
            F[b + p.nc] *= f;
            F[b + 2 * p.nc] *= f;
        }
        bad |= !isfinite(st.N[i]);
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

template <int G, typename P, bool R32>
__global__ void __launch_bounds__(kPass1Block)
thermo_pass1(ThermoParams p, const double *__restrict__ nH, double *xHII, double *xHeII, double *xHeIII,
             double *T, P *N, P *F, int32_t *subcycles, Queue q, unsigned *status)
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
        load_cell<G, false, P, R32>(p, c, xHII, xHeII, xHeIII, T, N, st, iso, cc);
        double n = nH[c];
        bool done = false;
        const int lim = p.pass1_attempts < p.max_sub ? p.pass1_attempts : p.max_sub;
        for (int k = 0; k < lim && !done; ++k)
            done = subcycle_once<G, false, R32>(p, n, st, t_left, dt_tc, att, iso, cc);
        if (!done && att >= p.max_sub) {
            atomicOr(status, kStatusSubcycle);
            done = true;
        }
        store_cell<G, P>(p, c, xHII, xHeII, xHeIII, T, N, F, st, status);
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

template <int G, typename P, bool R32>
__global__ void __launch_bounds__(128)
thermo_drain(ThermoParams p, const double *__restrict__ nH, double *xHII, double *xHeII, double *xHeIII,
             double *T, P *N, P *F, int32_t *subcycles, Queue q, DrainStage ds, unsigned *status)
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
            load_cell<G, false, P, R32>(p, c, xHII, xHeII, xHeIII, T, N, st, iso, cc);
            have = true;
        } else {
            have = false;
        }
    };
    fetch();
    while (have) {
        bool done = subcycle_once<G, false, R32>(p, n, st, t_left, dt_tc, att, iso, cc);
        if (!done && att >= p.max_sub) {
            atomicOr(status, kStatusSubcycle);
            done = true;
        }
        if (done) {
            store_cell<G, P>(p, c, xHII, xHeII, xHeIII, T, N, F, st, status);
            subcycles[c] = att;
            fetch();
        } else if (++used >= ds.budget) {
            // long sub-cycler: hand it to the next stage
            store_cell<G, P>(p, c, xHII, xHeII, xHeIII, T, N, F, st, status);
            unsigned long long slot = atomicAdd(&q.counters[ds.dst_cnt], 1ULL);
            push_item(ds.dst, slot, q.capacity, (uint32_t)c, t_left, dt_tc, att, status);
            fetch();
        }
    }
}

template <int G, typename P, bool R32>
__global__ void __launch_bounds__(128)
thermo_hard(ThermoParams p, const double *__restrict__ nH, double *xHII, double *xHeII, double *xHeIII,
            double *T, P *N, P *F, int32_t *subcycles, Queue q, unsigned *status)
{
    unsigned long long count = q.counters[4];
    if (count > (unsigned long long)q.capacity) count = (unsigned long long)q.capacity;
    if (count == 0) return;
    const int lane = threadIdx.x & 31;
    while (true) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(&q.counters[5], 1ULL);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= count) break;
        const long long c = q.a.cell[it];
        double t_left = q.a.t_left[it];
        double dt_tc = q.a.dt_tc[it];
        int att = q.a.attempts[it];
        const double n = nH[c];
        CellState<G> st;
        IsoRates<> iso;
        CoolCache<> cc;
        load_cell<G, true, P, R32>(p, c, xHII, xHeII, xHeIII, T, N, st, iso, cc);
        bool done = false;
        while (!done) {
            done = subcycle_once<G, true, R32>(p, n, st, t_left, dt_tc, att, iso, cc);
            if (!done && att >= p.max_sub) {
                if (lane == 0) atomicOr(status, kStatusSubcycle);
                done = true;
            }
        }
        if (lane == 0) {
            store_cell<G, P>(p, c, xHII, xHeII, xHeIII, T, N, F, st, status);
            subcycles[c] = att;
        }
        __syncwarp();
    }
}

template <int G, typename P, bool R32>
cudaError_t launch_g(const ThermoParams &tp, const double *nH, double *xHII, double *xHeII, double *xHeIII,
                     double *T, P *N, P *F, int32_t *sub, Queue q, unsigned *status, int n_sm,
                     cudaStream_t s, cudaEvent_t *ev)
{
    const int B = kPass1Block;
    long long nb = (tp.nc + B - 1) / B;
    if (ev) cudaEventRecord(ev[0], s);
    thermo_pass1<G, P, R32><<<(unsigned)nb, B, 0, s>>>(tp, nH, xHII, xHeII, xHeIII, T, N, F, sub, q, status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, thermo_drain<G, P, R32>, 128, 0);
        if (per_sm < 1) per_sm = 1;
    }
    long long grid = (long long)per_sm * n_sm;
    long long need = (tp.nc + 127) / 128;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    // one warp per long sub-cycler: two 4-warp blocks per SM
    long long hgrid = 2LL * n_sm;
    long long hneed = (tp.nc + 3) / 4;
    if (hgrid > hneed) hgrid = hneed;
    if (hgrid < 1) hgrid = 1;
    if (ev) { cudaEventRecord(ev[1], s); cudaEventRecord(ev[2], s); }
    DrainStage d1{q.a, q.b, 0, 2, kDrainBudget, 0};
    thermo_drain<G, P, R32><<<(unsigned)grid, 128, 0, s>>>(tp, nH, xHII, xHeII, xHeIII, T, N, F, sub, q, d1, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // many more long sub-cyclers than the warp-per-cell kernel has warps:
    // they share the FP64 pipes anyway, so a lane per cell does more per
    // cycle; up to twice its warps, the warps keep each cell's path short
    DrainStage d2{q.b, q.a, 2, 4, kDrain2Budget, 8 * hgrid};
    thermo_drain<G, P, R32><<<(unsigned)grid, 128, 0, s>>>(tp, nH, xHII, xHeII, xHeIII, T, N, F, sub, q, d2, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    thermo_hard<G, P, R32><<<(unsigned)hgrid, 128, 0, s>>>(tp, nH, xHII, xHeII, xHeIII, T, N, F, sub, q, status);
    if (ev) cudaEventRecord(ev[3], s);
    return cudaGetLastError();
}

}  // namespace

template <typename P, bool R32>
static cudaError_t dispatch_g(const ThermoParams &tp, int G, const double *nH, double *xHII, double *xHeII,
                              double *xHeIII, double *T, P *N, P *F, int32_t *sub, Queue q, unsigned *status,
                              int n_sm, cudaStream_t s, cudaEvent_t *ev)
{
    switch (G) {
    case 1: return launch_g<1, P, R32>(tp, nH, xHII, xHeII, xHeIII, T, N, F, sub, q, status, n_sm, s, ev);
    case 2: return launch_g<2, P, R32>(tp, nH, xHII, xHeII, xHeIII, T, N, F, sub, q, status, n_sm, s, ev);
    case 3: return launch_g<3, P, R32>(tp, nH, xHII, xHeII, xHeIII, T, N, F, sub, q, status, n_sm, s, ev);
    case 4: return launch_g<4, P, R32>(tp, nH, xHII, xHeII, xHeIII, T, N, F, sub, q, status, n_sm, s, ev);
    case 5: return launch_g<5, P, R32>(tp, nH, xHII, xHeII, xHeIII, T, N, F, sub, q, status, n_sm, s, ev);
    case 6: return launch_g<6, P, R32>(tp, nH, xHII, xHeII, xHeIII, T, N, F, sub, q, status, n_sm, s, ev);
    case 7: return launch_g<7, P, R32>(tp, nH, xHII, xHeII, xHeIII, T, N, F, sub, q, status, n_sm, s, ev);
    case 8: return launch_g<8, P, R32>(tp, nH, xHII, xHeII, xHeIII, T, N, F, sub, q, status, n_sm, s, ev);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_thermo(const ThermoParams &tp, int G, const double *nH, double *xHII, double *xHeII,
                          double *xHeIII, double *T, double *N, double *F, int32_t *subcycles, Queue q,
                          unsigned *status, int n_sm, cudaStream_t s, cudaEvent_t *ev)
{
    return dispatch_g<double, false>(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, subcycles, q, status, n_sm, s, ev);
}

cudaError_t launch_thermo_mixed(const ThermoParams &tp, int G, bool rates32, const double *nH, double *xHII,
                                double *xHeII, double *xHeIII, double *T, float *N, float *F, int32_t *subcycles,
                                Queue q, unsigned *status, int n_sm, cudaStream_t s, cudaEvent_t *ev)
{
    if (rates32)
        return dispatch_g<float, true>(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, subcycles, q, status, n_sm, s, ev);
    return dispatch_g<float, false>(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, subcycles, q, status, n_sm, s, ev);
}

}  // namespace rtgb

// ---------------------------------------------------------------------------
// Allocation-free thermochemistry entry point (rt_thermo_step_noalloc).
//
// For callers that cannot allocate device memory at call time: the work
// queue lives in a fixed file-scope device array instead of memory owned by
// an rt_handle.  Every GPU that loads the library holds this array until
// the process exits.  All calls share it, and its contents persist from the
// previous call, so the queue counters and the status word are cleared at
// the start of every call; calls whose kernels overlap on the GPU race on
// it and must not be issued.
namespace rtgb {
namespace {

constexpr long long kNoAllocMaxCells = 1LL << 18;   // 262144 cells
// layout: [0,64) queue counters, [64,68) status; from byte 256 the two
// queues, each cell / attempts / t_left / dt_tc arrays of kNoAllocMaxCells
constexpr size_t kNoAllocHeader = 256;
constexpr size_t kNoAllocQueueBytes =
    (size_t)kNoAllocMaxCells * (sizeof(uint32_t) + sizeof(int32_t) + 2 * sizeof(double));
constexpr size_t kNoAllocBytes = kNoAllocHeader + 2 * kNoAllocQueueBytes;

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_addr[kMaxDevices] = {};

}  // namespace

static __device__ __align__(256) unsigned char g_thermo_scratch[kNoAllocBytes];

namespace {

// Device address of g_thermo_scratch on the current device, looked up once
// per device.  In host code the symbol names a host-side shadow, so only
// this address may be handed to kernels.
cudaError_t noalloc_scratch(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_thermo_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

}  // namespace

}  // namespace rtgb

extern "C" int rt_thermo_step_noalloc(long long ncells, int n_groups, const rt_options *opt, double c_r,
                                      const double *sigN, const double *sigE, const double *egy, double dt,
                                      const double *nH, double *xHII, double *xHeII, double *xHeIII, double *T,
                                      double *N, double *F, int32_t *subcycles, void *stream)
{
    using namespace rtgb;
    if (ncells < 1 || ncells > kNoAllocMaxCells) return RT_EINVAL;
    if (n_groups < 1 || n_groups > RT_MAX_GROUPS || !opt || !sigN || !sigE || !egy) return RT_EINVAL;
    if (!nH || !xHII || !xHeII || !xHeIII || !T || !N || !F || !subcycles) return RT_EINVAL;
    if (!(c_r > 0.0) || !(dt > 0.0) || !(opt->X > 0.0 && opt->X <= 1.0)) return RT_EINVAL;
    if (opt->otsa != 1 || opt->smooth != 0 || opt->precision != RT_FP64 || opt->max_subcycles < 1 ||
        !(opt->a_exp > 0.0))
        return RT_EINVAL;
    for (int i = 0; i < 3 * n_groups; ++i)
        if (!(sigN[i] >= 0.0) || !(sigE[i] >= 0.0)) return RT_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, n_sm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess) return RT_ECUDA;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return RT_ECUDA;
    unsigned char *base = nullptr;
    if (noalloc_scratch(dev, &base) != cudaSuccess) return RT_ECUDA;

    ThermoParams tp{};
    tp.nc = ncells;
    tp.dt = dt;
    tp.cr = c_r;
    tp.X = opt->X;
    const double Y = 1.0 - opt->X;
    tp.he_ratio = (Y > 0.0) ? Y / (4.0 * opt->X) : 0.0;
    tp.kfac = (5.0 / 3.0 - 1.0) * opt->X / 1.380649e-16;
    tp.a_exp = opt->a_exp;
    tp.isothermal = opt->isothermal ? 1 : 0;
    tp.helium = (Y > 0.0) ? 1 : 0;
    tp.case_b = 1;
    tp.max_sub = opt->max_subcycles;
    tp.pass1_attempts = 6;
    for (int i = 0; i < n_groups; ++i) {
        for (int j = 0; j < 3; ++j) {
            tp.gc.sigN[i][j] = sigN[3 * i + j];
            tp.gc.sigE[i][j] = sigE[3 * i + j];
        }
        tp.gc.egy[i] = egy[i];
    }
    Queue q{};
    q.counters = reinterpret_cast<unsigned long long *>(base);
    unsigned *status = reinterpret_cast<unsigned *>(base + 8 * kQueueCounters);
    const size_t K = (size_t)kNoAllocMaxCells;
    QueueArrays *qa[2] = {&q.a, &q.b};
    for (int k = 0; k < 2; ++k) {
        unsigned char *qb = base + kNoAllocHeader + k * kNoAllocQueueBytes;
        qa[k]->cell = reinterpret_cast<uint32_t *>(qb);
        qa[k]->attempts = reinterpret_cast<int32_t *>(qb + 4 * K);
        qa[k]->t_left = reinterpret_cast<double *>(qb + 8 * K);
        qa[k]->dt_tc = reinterpret_cast<double *>(qb + 16 * K);
    }
    q.capacity = ncells;

    if (cudaMemsetAsync(base, 0, kNoAllocHeader, s) != cudaSuccess) return RT_ECUDA;
    if (launch_thermo(tp, n_groups, nH, xHII, xHeII, xHeIII, T, N, F, subcycles, q, status, n_sm, s) !=
        cudaSuccess)
        return RT_ECUDA;
    unsigned st = 0;
    if (cudaMemcpyAsync(&st, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RT_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return RT_ECUDA;
    if (st & kStatusNonFinite) return RT_ENONFINITE;
    if (st & kStatusSubcycle) return RT_ESUBCYCLE;
    if (st & kStatusQueue) return RT_EQUEUE;
    return RT_OK;
}

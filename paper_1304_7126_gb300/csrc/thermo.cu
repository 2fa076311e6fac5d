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
//                 ThermoParams::drain_budget attempts here moves to queue B
//                 (a second stage with its own budget runs when queue B is
//                 long);
//   thermo_hard   persistent; a pair of warps per queue-C cell.  On GB300
//                 a lone dependent chain is slow (64 cycles per FP64 FMA),
//                 so the lanes of a warp evaluate the cell's rate and
//                 cooling functions of one temperature in parallel (rates.cuh,
//                 one lane each) while the scalar update runs redundantly in
//                 all lanes, and the second warp of the pair computes the
//                 cooling while the first updates the photons.  The
//                 arithmetic is identical to the one-thread path, and a
//                 queued cell carries its flux scale, so results do not
//                 depend on which kernel finished a cell.
// Nothing waits on another thread; each kernel ends when its queue is empty.
// The kernels live in thermo_kernels.cuh, instantiated per precision family
// in thermo_f64.cu, thermo_mix.cu, thermo_mix32.cu and their smoothed-RT
// counterparts (*_sm.cu); this file holds the launchers and the
// allocation-free entry point.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "rt_internal.h"

namespace rtgb {

cudaError_t launch_thermo(const ThermoParams &tp, int G, const double *nH, double *xHII, double *xHeII,
                          double *xHeIII, double *T, double *N, double *F, double *Npre, double *Fpre,
                          int32_t *subcycles, Queue q, unsigned *status, int n_sm, cudaStream_t s, cudaEvent_t *ev)
{
    if (Npre)
        return thermo_dispatch_f64_sm(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, subcycles, q, status, n_sm,
                                      s, ev);
    return thermo_dispatch_f64(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, nullptr, nullptr, subcycles, q, status, n_sm, s,
                               ev);
}

cudaError_t launch_thermo_mixed(const ThermoParams &tp, int G, bool rates32, const double *nH, double *xHII,
                                double *xHeII, double *xHeIII, double *T, float *N, float *F, float *Npre,
                                float *Fpre, int32_t *subcycles, Queue q, unsigned *status, int n_sm, cudaStream_t s,
                                cudaEvent_t *ev)
{
    if (rates32) {
        if (Npre)
            return thermo_dispatch_mix32_sm(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, subcycles, q, status,
                                            n_sm, s, ev);
        return thermo_dispatch_mix32(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, nullptr, nullptr, subcycles, q, status,
                                     n_sm, s, ev);
    }
    if (Npre)
        return thermo_dispatch_mix_sm(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, Npre, Fpre, subcycles, q, status, n_sm,
                                      s, ev);
    return thermo_dispatch_mix(tp, G, nH, xHII, xHeII, xHeIII, T, N, F, nullptr, nullptr, subcycles, q, status, n_sm, s,
                               ev);
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
// queues, each cell / attempts / t_left / dt_tc arrays of kNoAllocMaxCells,
// then the queued cells' flux scales, RT_MAX_GROUPS x kNoAllocMaxCells doubles
constexpr size_t kNoAllocHeader = 256;
constexpr size_t kNoAllocQueueBytes =
    (size_t)kNoAllocMaxCells * (sizeof(uint32_t) + sizeof(int32_t) + 2 * sizeof(double));
constexpr size_t kNoAllocScaleBytes = (size_t)kNoAllocMaxCells * RT_MAX_GROUPS * sizeof(double);
constexpr size_t kNoAllocBytes = kNoAllocHeader + 2 * kNoAllocQueueBytes + kNoAllocScaleBytes;

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_addr[kMaxDevices] = {};
unsigned long long g_noalloc_ctx[kMaxDevices] = {};   // context id the address belongs to

}  // namespace

static __device__ __align__(256) unsigned char g_thermo_scratch[kNoAllocBytes];

namespace {

// Id of the current context (the driver's cuCtxGetCurrent and cuCtxGetId,
// reached through the runtime so the library needs no link to the driver
// library).  A device reset replaces the primary context, and with it the
// module that holds g_thermo_scratch; the id tells the two apart.
cudaError_t current_context_id(unsigned long long *id)
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    if (!get_current || !get_id) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb);
        if (e != cudaSuccess) return e;
        if (qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
            return cudaErrorNotSupported;
        get_current = reinterpret_cast<GetCurrent>(a);
        get_id = reinterpret_cast<GetId>(b);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
    if (get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorUnknown;
    return cudaSuccess;
}

// Device address of g_thermo_scratch on the current device, looked up once
// per device and context (again after a device reset).  In host code the
// symbol names a host-side shadow, so only this address may be handed to
// kernels.
cudaError_t noalloc_scratch(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    unsigned long long ctx = 0;
    cudaError_t e = current_context_id(&ctx);
    if (e != cudaSuccess || !g_noalloc_addr[dev] || g_noalloc_ctx[dev] != ctx) {
        // (the lookup also creates the primary context if there is none yet)
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_thermo_scratch);
        if (e != cudaSuccess) return e;
        e = current_context_id(&ctx);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = static_cast<unsigned char *>(p);
        g_noalloc_ctx[dev] = ctx;
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
    // the option and constant checks of rt_create, and a finite dt > 0
    if (!(c_r > 0.0) || !std::isfinite(c_r) || !(dt > 0.0) || !std::isfinite(dt)) return RT_EINVAL;
    if (!(opt->X > 0.0 && opt->X <= 1.0)) return RT_EINVAL;
    if (opt->otsa != 1 || opt->smooth != 0 || opt->precision != RT_FP64 || opt->max_subcycles < 1 ||
        !(opt->a_exp > 0.0) || !std::isfinite(opt->a_exp))
        return RT_EINVAL;
    for (int i = 0; i < 3 * n_groups; ++i)
        if (!(sigN[i] >= 0.0) || !(sigE[i] >= 0.0) || !std::isfinite(sigN[i]) || !std::isfinite(sigE[i]))
            return RT_EINVAL;
    for (int i = 0; i < n_groups; ++i)
        if (!(egy[i] > 0.0) || !std::isfinite(egy[i])) return RT_EINVAL;
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
    default_routing(tp);
    for (int i = 0; i < n_groups; ++i) {
        for (int j = 0; j < 3; ++j) {
            tp.gc.sigN[i][j] = sigN[3 * i + j];
            tp.gc.sigE[i][j] = sigE[3 * i + j];
        }
        tp.gc.egy[i] = egy[i];
    }
    derive_group_terms(tp);
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
    q.fscale = reinterpret_cast<double *>(base + kNoAllocHeader + 2 * kNoAllocQueueBytes);

    if (cudaMemsetAsync(base, 0, kNoAllocHeader, s) != cudaSuccess) return RT_ECUDA;
    if (launch_thermo(tp, n_groups, nH, xHII, xHeII, xHeIII, T, N, F, nullptr, nullptr, subcycles, q, status, n_sm,
                      s) !=
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

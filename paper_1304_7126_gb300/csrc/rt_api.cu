// C-ABI of the rtgb library (declared in include/rt.h): handle lifetime,
// state transfer, source list, and the RT step (paper Sec. 3: injection,
// transport, thermochemistry over the same dt), optionally replayed as a
// CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "rt_internal.h"
#include "state_check.h"

using namespace rtgb;

struct rt_handle {
    GridDev g{};
    int G = 0;
    rt_options opt{};
    double cr = 0.0;
    GroupConsts gc{};
    int device = 0;
    int n_sm = 1;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;

    double *nH = nullptr, *xHII = nullptr, *xHeII = nullptr, *xHeIII = nullptr, *T = nullptr;
    double *N[2] = {nullptr, nullptr};   // RT_FP64 photon state
    double *F[2] = {nullptr, nullptr};
    float *Nf[2] = {nullptr, nullptr};   // RT_MIXED photon state
    float *Ff[2] = {nullptr, nullptr};
    void *Npre = nullptr, *Fpre = nullptr;   // smoothed RT: photon state before injection
    double *inflow_d = nullptr;              // [G][6][4] ghost states of inflow faces
    float *inflow_f = nullptr;
    bool mixed = false;
    int cur = 0;
    double *hll = nullptr;
    float *hllf = nullptr;
    int32_t *subcycles = nullptr;
    Queue q{};
    Partials part{};
    double *budget = nullptr;
    unsigned *status = nullptr;
    unsigned *status_host = nullptr;   // pinned mirror, refreshed after every step

    int nsrc = 0;
    long long *src_cell = nullptr;
    double *src_L = nullptr;
    std::vector<double> src_Lsum_host;   // total luminosity per group
    int nsrc_orig = 0;                    // sources as given (not merged per cell)
    long long *src_cell_orig = nullptr;

    // adjoint scratch (rt_step_vjp, rt_run_vjp)
    double *adj = nullptr;               // NA, FA, NB, FB, lNb, lFb, gas copy
    int32_t *adj_sub = nullptr;          // [2][nc] attempts: adjoint, forward check
    unsigned long long *adj_count = nullptr;

    bool state_set = false;
    ThermoParams routing{};   // only the routing fields are used (rt_set_thermo_routing)
    cudaGraphExec_t graph = nullptr;
    double graph_dt = 0.0;
    int graph_cur0 = 0;     // ping-pong buffer the captured pair of steps starts from
    std::string err;

    // per-phase profiling (rt_set_profiling)
    bool prof = false;
    cudaEvent_t ev[RT_NPHASES + 1][2] = {};
    bool ev_made = false;
    double prof_ms[RT_NPHASES] = {0};
    int64_t prof_n[RT_NPHASES] = {0};
    std::vector<cudaEvent_t> pending;   // [start, stop] pairs per phase, flattened
    std::vector<int> pending_phase;
};

namespace {

const char *kNoHandle = "null handle";

int fail(rt_handle *h, int code, const std::string &msg)
{
    if (h) h->err = msg;
    return code;
}

int cuda_fail(rt_handle *h, cudaError_t e, const char *what)
{
    return fail(h, RT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define RT_CUDA(h, call)                                  \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

double courant(const rt_handle *h) { return h->opt.cfl * h->g.dx / (3.0 * h->cr); }

int status_to_code(rt_handle *h, unsigned st)
{
    if (st & kStatusNonFinite) return fail(h, RT_ENONFINITE, "non-finite value in the state");
    if (st & kStatusSubcycle) return fail(h, RT_ESUBCYCLE, "a cell exceeded max_subcycles thermochemistry attempts");
    if (st & kStatusQueue) return fail(h, RT_EQUEUE, "thermochemistry work queue overflow");
    return RT_OK;
}

void prof_collect(rt_handle *h);

int sync_and_check(rt_handle *h)
{
    RT_CUDA(h, cudaStreamSynchronize(h->stream));
    prof_collect(h);
    unsigned st = 0;
    RT_CUDA(h, cudaMemcpy(&st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    return status_to_code(h, st);
}

void free_all(rt_handle *h)
{
    if (h->graph) cudaGraphExecDestroy(h->graph);
    for (cudaEvent_t e : h->pending) cudaEventDestroy(e);
    h->pending.clear();
    void *ptrs[] = {h->nH, h->xHII, h->xHeII, h->xHeIII, h->T, h->N[0], h->N[1], h->F[0], h->F[1],
                    h->Nf[0], h->Nf[1], h->Ff[0], h->Ff[1], h->hllf, h->hll, h->subcycles, h->q.a.cell, h->q.a.t_left, h->q.a.dt_tc, h->q.a.attempts,
                    h->q.b.cell, h->q.b.t_left, h->q.b.dt_tc, h->q.b.attempts, h->q.counters, h->q.fscale, h->part.tr_inbox, h->part.tr_outflow, h->part.th_inbox,
                    h->budget, h->status, h->src_cell, h->src_L, h->src_cell_orig, h->adj, h->adj_sub, h->Npre, h->Fpre, h->inflow_d, h->inflow_f,
                    h->adj_count};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->status_host) cudaFreeHost(h->status_host);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
}

template <typename T>
int dalloc(rt_handle *h, T **p, size_t n)
{
    cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return fail(h, RT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return RT_OK;
}

ThermoParams thermo_params(const rt_handle *h, double dt)
{
    ThermoParams p{};
    p.nc = h->g.nc;
    p.dt = dt;
    p.cr = h->cr;
    p.X = h->opt.X;
    double Y = 1.0 - h->opt.X;
    p.he_ratio = (Y > 0.0) ? Y / (4.0 * h->opt.X) : 0.0;
    // K = (gamma - 1) m_H / (rho k_B) with rho = n_H m_H / X
    p.kfac = (5.0 / 3.0 - 1.0) * h->opt.X / 1.380649e-16;
    p.a_exp = h->opt.a_exp;
    p.isothermal = h->opt.isothermal ? 1 : 0;
    p.helium = (Y > 0.0) ? 1 : 0;
    p.case_b = h->opt.otsa ? 1 : 0;
    p.max_sub = h->opt.max_subcycles;
    p.pass1_attempts = h->routing.pass1_attempts;
    p.drain_budget = h->routing.drain_budget;
    p.drain2_budget = h->routing.drain2_budget;
    p.drain2_min = h->routing.drain2_min;
    p.emit = h->opt.otsa ? 0 : 1;
    for (int j = 0; j < 3; ++j) {
        int r = h->opt.rec_group[j];
        p.rec_g[j] = (r == RT_REC_BY_BAND) ? std::min(j, h->G - 1) : r;
    }
    p.gc = h->gc;
    derive_group_terms(p);
    return p;
}

// Profiling: a fresh start/stop event pair per phase launch; elapsed times
// are folded in at the next synchronising call.
void prof_pair(rt_handle *h, int phase, cudaEvent_t *a, cudaEvent_t *b)
{
    cudaEventCreate(a);
    cudaEventCreate(b);
    h->pending.push_back(*a);
    h->pending.push_back(*b);
    h->pending_phase.push_back(phase);
}

void prof_collect(rt_handle *h)
{
    for (size_t k = 0; k < h->pending_phase.size(); ++k) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, h->pending[2 * k], h->pending[2 * k + 1]) == cudaSuccess) {
            h->prof_ms[h->pending_phase[k]] += ms;
            h->prof_n[h->pending_phase[k]] += 1;
        }
        cudaEventDestroy(h->pending[2 * k]);
        cudaEventDestroy(h->pending[2 * k + 1]);
    }
    h->pending.clear();
    h->pending_phase.clear();
}

// Enqueue one RT step on h->stream (no host synchronisation).
int enqueue_step(rt_handle *h, double dt, bool capturing = false)
{
    const bool prof = h->prof && !capturing;
    cudaEvent_t a, b;
    const long long nc = h->g.nc;
    const double V = h->g.dx * h->g.dx * h->g.dx;
    cudaError_t e;
    if (h->opt.smooth) {
        // smoothed RT (Sec. 3.4): keep the state before injection and transport
        const size_t es = h->mixed ? sizeof(float) : sizeof(double);
        const void *n0 = h->mixed ? (const void *)h->Nf[h->cur] : (const void *)h->N[h->cur];
        const void *f0 = h->mixed ? (const void *)h->Ff[h->cur] : (const void *)h->F[h->cur];
        e = cudaMemcpyAsync(h->Npre, n0, es * h->G * nc, cudaMemcpyDeviceToDevice, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->Fpre, f0, es * 3 * h->G * nc, cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "smoothing copy");
    }
    if (h->nsrc > 0) {
        if (prof) { prof_pair(h, 0, &a, &b); cudaEventRecord(a, h->stream); }
        if (h->mixed) e = launch_inject_f32(h->nsrc, h->G, nc, h->src_cell, h->src_L, dt / V, h->Nf[h->cur], h->stream);
        else e = launch_inject(h->nsrc, h->G, nc, h->src_cell, h->src_L, dt / V, h->N[h->cur], h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "inject");
        if (prof) cudaEventRecord(b, h->stream);
    }
    int nxt = 1 - h->cur;
    if (prof) { prof_pair(h, 1, &a, &b); cudaEventRecord(a, h->stream); }
    if (h->mixed)
        e = launch_transport_f32(h->g, h->G, h->opt.flux, h->cr, dt, h->Nf[h->cur], h->Ff[h->cur], h->Nf[nxt],
                                 h->Ff[nxt], h->hllf, h->inflow_f, h->part, h->stream);
    else
        e = launch_transport(h->g, h->G, h->opt.flux, h->cr, dt, h->N[h->cur], h->F[h->cur], h->N[nxt],
                             h->F[nxt], h->hll, h->inflow_d, h->part, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "transport");
    if (prof) cudaEventRecord(b, h->stream);
    h->cur = nxt;
    ThermoParams tp = thermo_params(h, dt);
    cudaEvent_t tev[4];
    if (prof) {
        prof_pair(h, 2, &tev[0], &tev[1]);
        prof_pair(h, 3, &tev[2], &tev[3]);
    }
    if (h->mixed)
        e = launch_thermo_mixed(tp, h->G, h->opt.precision == RT_MIXED32, h->nH, h->xHII, h->xHeII, h->xHeIII, h->T,
                                h->Nf[h->cur], h->Ff[h->cur], (float *)h->Npre, (float *)h->Fpre, h->subcycles, h->q,
                                h->status, h->n_sm, h->stream, prof ? tev : nullptr);
    else
        e = launch_thermo(tp, h->G, h->nH, h->xHII, h->xHeII, h->xHeIII, h->T, h->N[h->cur], h->F[h->cur],
                          (double *)h->Npre, (double *)h->Fpre, h->subcycles, h->q, h->status, h->n_sm, h->stream,
                          prof ? tev : nullptr);
    if (e != cudaSuccess) return cuda_fail(h, e, "thermo");
    if (prof) { prof_pair(h, 4, &a, &b); cudaEventRecord(a, h->stream); }
    e = h->mixed ? launch_reduce_N_f32(h->G, nc, h->Nf[h->cur], h->part, h->stream)
                 : launch_reduce_N(h->G, nc, h->N[h->cur], h->part, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reduce");
    if (prof) cudaEventRecord(b, h->stream);
    double emitted[kMaxG] = {0};
    for (int g = 0; g < h->G; ++g) emitted[g] = h->src_Lsum_host[g] * dt;
    if (prof) { prof_pair(h, 5, &a, &b); cudaEventRecord(a, h->stream); }
    e = launch_finalize_mode(h->G, 0, h->part, V, emitted, h->budget, h->q, h->status, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "finalize");
    if (prof) cudaEventRecord(b, h->stream);
    e = cudaMemcpyAsync(h->status_host, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "status copy");
    return RT_OK;
}

int check_dt(rt_handle *h, double *dt)
{
    if (!h->state_set) return fail(h, RT_EINVAL, "rt_set_state has not been called");
    double dc = courant(h);
    if (!(*dt > 0.0)) *dt = dc;
    if (!std::isfinite(*dt)) return fail(h, RT_EINVAL, "dt is not finite");
    if (*dt > dc * (1.0 + 1e-12)) return fail(h, RT_EDT, "dt above the Courant limit CFL dx/(3 c_r)");
    // the pinned mirror of the sticky status (stale by at most the steps in flight)
    unsigned st = *(volatile unsigned *)h->status_host;
    if (st) return status_to_code(h, st);
    return RT_OK;
}

void invalidate_graph(rt_handle *h)
{
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
}


int ensure_adj(rt_handle *h)
{
    if (h->adj) return RT_OK;
    const long long nc = h->g.nc;
    int rc;
    if ((rc = dalloc(h, &h->adj, (size_t)(12 * h->G + 4) * nc)) || (rc = dalloc(h, &h->adj_sub, 2 * (size_t)nc)) ||
        (rc = dalloc(h, &h->adj_count, 1)))
        return rc;
    return RT_OK;
}

// Adjoint of one step from the handle's state U_k (left unchanged); see
// rt_step_vjp.  check: also re-run the forward thermochemistry on a copy of
// U_b and count the cells whose attempt count differs from the adjoint's
// recomputation into adj_count.
int enqueue_vjp(rt_handle *h, double dt, double *lx, double *ly2, double *ly3, double *lT, double *lN,
                double *lF, double *g_nH, double *g_L, bool check)
{
    const long long nc = h->g.nc;
    const int G = h->G;
    const double V = h->g.dx * h->g.dx * h->g.dx;
    int rc = ensure_adj(h);
    if (rc) return rc;
    double *NA = h->adj, *FA = NA + G * nc, *NB = FA + 3 * G * nc, *FB = NB + G * nc;
    double *lNb = FB + 3 * G * nc, *lFb = lNb + G * nc, *gas = lFb + 3 * G * nc;
    cudaStream_t st = h->stream;
    const int c0 = h->cur;
    cudaError_t e;
    RT_CUDA(h, cudaMemcpyAsync(NA, h->N[c0], G * nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
    RT_CUDA(h, cudaMemcpyAsync(FA, h->F[c0], 3 * G * nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (h->nsrc > 0) {
        e = launch_inject(h->nsrc, G, nc, h->src_cell, h->src_L, dt / V, NA, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "inject");
    }
    e = launch_transport(h->g, G, h->opt.flux, h->cr, dt, NA, FA, NB, FB, h->hll, h->inflow_d, h->part, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "transport");
    ThermoParams tp = thermo_params(h, dt);
    int32_t *sub_adj = check ? h->adj_sub : nullptr;
    e = launch_thermo_vjp(tp, G, h->nH, h->xHII, h->xHeII, h->xHeIII, h->T, NB, FB, lx, ly2, ly3, lT, lN, lF, lNb,
                          lFb, g_nH, sub_adj, h->status, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "thermo_vjp");
    e = launch_clamp_vjp(G, nc, h->cr, NB, FB, lNb, lFb, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "clamp_vjp");
    e = launch_transport_vjp(h->g, G, h->opt.flux, h->cr, dt, NA, FA, h->hll, h->inflow_d, lNb, lFb, lN, lF, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "transport_vjp");
    e = launch_inject_vjp(h->nsrc_orig, G, nc, h->src_cell_orig, lN, dt / V, g_L, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "inject_vjp");
    if (check) {
        double *gx = gas, *gy2 = gas + nc, *gy3 = gas + 2 * nc, *gT = gas + 3 * nc;
        RT_CUDA(h, cudaMemcpyAsync(gx, h->xHII, nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
        RT_CUDA(h, cudaMemcpyAsync(gy2, h->xHeII, nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
        RT_CUDA(h, cudaMemcpyAsync(gy3, h->xHeIII, nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
        RT_CUDA(h, cudaMemcpyAsync(gT, h->T, nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
        e = launch_thermo(tp, G, h->nH, gx, gy2, gy3, gT, NB, FB, nullptr, nullptr, h->adj_sub + nc, h->q, h->status,
                          h->n_sm, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "thermo");
        RT_CUDA(h, cudaMemsetAsync(h->q.counters, 0, kQueueCounters * sizeof(unsigned long long), st));
        e = launch_count_mismatch(nc, h->adj_sub, h->adj_sub + nc, h->adj_count, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "count");
    }
    return RT_OK;
}

int vjp_args(rt_handle *h, double *dt, double *lx, double *ly2, double *ly3, double *lT, double *lN, double *lF,
             double *g_nH, double *g_L)
{
    if (h->opt.precision != RT_FP64 || h->opt.smooth || !h->opt.otsa)
        return fail(h, RT_EINVAL, "the adjoint needs precision RT_FP64, the OTSA and no smoothing");
    if (!lx || !ly2 || !ly3 || !lT || !lN || !lF || !g_nH || (h->nsrc_orig > 0 && !g_L))
        return fail(h, RT_EINVAL, "null adjoint array");
    return check_dt(h, dt);
}

}  // namespace

extern "C" {

void rt_default_options(rt_options *o)
{
    if (!o) return;
    o->X = 0.76;
    o->isothermal = 0;
    o->otsa = 1;
    o->flux = RT_GLF;
    o->cfl = 0.8;
    o->precision = RT_FP64;
    o->a_exp = 1.0;
    o->max_subcycles = 1000000;
    o->smooth = 0;
    o->rec_group[0] = o->rec_group[1] = o->rec_group[2] = RT_REC_BY_BAND;
}

int rt_version(void) { return 100; }

int rt_hll_table(int nf, int nmu, double *out)
{
    if (nf < 2 || nmu < 2 || !out) return RT_EINVAL;
    rtgb::hll_table(nf, nmu, out);
    return RT_OK;
}

int rt_create(const rt_grid *grid, int n_groups, const rt_options *opt, double c_r, const double *sigN,
              const double *sigE, const double *egy, rt_handle **out)
{
    if (!out) return RT_EINVAL;
    *out = nullptr;
    if (!grid || !opt || !sigN || !sigE || !egy) return RT_EINVAL;
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->dx_cm > 0.0) || !std::isfinite(grid->dx_cm))
        return RT_EINVAL;
    long long nc = (long long)grid->nx * grid->ny * grid->nz;
    if (nc >= (1LL << 31)) return RT_EINVAL;
    for (int i = 0; i < 6; ++i)
        if (grid->bc[i] < RT_BC_OUTFLOW || grid->bc[i] > RT_BC_INFLOW) return RT_EINVAL;
    for (int d = 0; d < 3; ++d)   // periodic must be set on both faces of an axis
        if ((grid->bc[2 * d] == RT_BC_PERIODIC) != (grid->bc[2 * d + 1] == RT_BC_PERIODIC)) return RT_EINVAL;
    if (n_groups < 1 || n_groups > RT_MAX_GROUPS) return RT_EINVAL;
    if (!(c_r > 0.0) || !std::isfinite(c_r)) return RT_EINVAL;
    if (!(opt->X > 0.0 && opt->X <= 1.0)) return RT_EINVAL;
    if (!(opt->cfl > 0.0 && opt->cfl <= 1.0)) return RT_EINVAL;
    if (opt->flux != RT_GLF && opt->flux != RT_HLL) return RT_EINVAL;
    if ((opt->otsa != 0 && opt->otsa != 1) || (opt->smooth != 0 && opt->smooth != 1)) return RT_EINVAL;
    for (int j = 0; j < 3; ++j)
        if (opt->rec_group[j] != RT_REC_BY_BAND && (opt->rec_group[j] < -1 || opt->rec_group[j] >= n_groups))
            return RT_EINVAL;
    if (opt->precision != RT_FP64 && opt->precision != RT_MIXED && opt->precision != RT_MIXED32) return RT_EINVAL;
    if (!(opt->a_exp > 0.0) || !std::isfinite(opt->a_exp) || opt->max_subcycles < 1) return RT_EINVAL;
    for (int i = 0; i < 3 * n_groups; ++i)
        if (!(sigN[i] >= 0.0) || !(sigE[i] >= 0.0) || !std::isfinite(sigN[i]) || !std::isfinite(sigE[i]))
            return RT_EINVAL;
    for (int i = 0; i < n_groups; ++i)
        if (!(egy[i] > 0.0) || !std::isfinite(egy[i])) return RT_EINVAL;

    rt_handle *h = new rt_handle();
    default_routing(h->routing);
    h->g.nx = grid->nx; h->g.ny = grid->ny; h->g.nz = grid->nz;
    h->g.nc = nc;
    h->g.stride = nc;
    h->g.dx = grid->dx_cm;
    for (int i = 0; i < 6; ++i) h->g.bc[i] = grid->bc[i];
    h->G = n_groups;
    h->opt = *opt;
    h->mixed = opt->precision == RT_MIXED || opt->precision == RT_MIXED32;
    h->cr = c_r;
    for (int i = 0; i < n_groups; ++i) {
        for (int j = 0; j < 3; ++j) {
            h->gc.sigN[i][j] = sigN[3 * i + j];
            h->gc.sigE[i][j] = sigE[3 * i + j];
        }
        h->gc.egy[i] = egy[i];
    }
    h->src_Lsum_host.assign(n_groups, 0.0);
    int rc = RT_OK;
    cudaError_t e;
    if ((e = cudaGetDevice(&h->device)) != cudaSuccess) { rc = cuda_fail(h, e, "cudaGetDevice"); goto bad; }
    if ((e = cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->device)) != cudaSuccess) {
        rc = cuda_fail(h, e, "attr"); goto bad;
    }
    if ((e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        rc = cuda_fail(h, e, "cudaStreamCreate"); goto bad;
    }
    h->stream = h->own_stream;
    transport_init();
    {
        const size_t G = (size_t)n_groups;
        h->part.n_tr_blocks = transport_grid(h->n_sm, h->mixed);
        h->part.n_red_blocks = reduce_blocks_per_group();
        if ((rc = dalloc(h, &h->nH, nc)) || (rc = dalloc(h, &h->xHII, nc)) || (rc = dalloc(h, &h->xHeII, nc)) ||
            (rc = dalloc(h, &h->xHeIII, nc)) || (rc = dalloc(h, &h->T, nc)) ||
            (rc = dalloc(h, &h->hll, (size_t)kHllNF * kHllNMU * 2)) || (rc = dalloc(h, &h->subcycles, nc)) ||
            (rc = dalloc(h, &h->q.a.cell, nc)) || (rc = dalloc(h, &h->q.a.t_left, nc)) ||
            (rc = dalloc(h, &h->q.a.dt_tc, nc)) || (rc = dalloc(h, &h->q.a.attempts, nc)) ||
            (rc = dalloc(h, &h->q.b.cell, nc)) || (rc = dalloc(h, &h->q.b.t_left, nc)) ||
            (rc = dalloc(h, &h->q.b.dt_tc, nc)) || (rc = dalloc(h, &h->q.b.attempts, nc)) ||
            (rc = dalloc(h, &h->q.counters, kQueueCounters)) ||
            (rc = dalloc(h, &h->q.fscale, (opt->smooth ? 2 : 1) * G * nc)) ||
            (rc = dalloc(h, &h->part.tr_inbox, G * h->part.n_tr_blocks)) ||
            (rc = dalloc(h, &h->part.tr_outflow, G * h->part.n_tr_blocks)) ||
            (rc = dalloc(h, &h->part.th_inbox, G * h->part.n_red_blocks)) ||
            (rc = dalloc(h, &h->budget, 4 * G)) || (rc = dalloc(h, &h->status, 1)))
            goto bad;
        for (int k = 0; k < 2; ++k) {
            if (h->mixed) {
                if ((rc = dalloc(h, &h->Nf[k], G * nc)) || (rc = dalloc(h, &h->Ff[k], 3 * G * nc))) goto bad;
                cudaMemset(h->Nf[k], 0, G * nc * sizeof(float));
                cudaMemset(h->Ff[k], 0, 3 * G * nc * sizeof(float));
            } else {
                if ((rc = dalloc(h, &h->N[k], G * nc)) || (rc = dalloc(h, &h->F[k], 3 * G * nc))) goto bad;
                cudaMemset(h->N[k], 0, G * nc * sizeof(double));
                cudaMemset(h->F[k], 0, 3 * G * nc * sizeof(double));
            }
        }
        if ((rc = dalloc(h, &h->inflow_d, (size_t)24 * G))) goto bad;
        cudaMemset(h->inflow_d, 0, 24 * G * sizeof(double));
        if (h->mixed) {
            if ((rc = dalloc(h, &h->inflow_f, (size_t)24 * G))) goto bad;
            cudaMemset(h->inflow_f, 0, 24 * G * sizeof(float));
        }
        if (opt->smooth) {
            const size_t es = h->mixed ? sizeof(float) : sizeof(double);
            if ((e = cudaMalloc(&h->Npre, es * G * nc)) != cudaSuccess ||
                (e = cudaMalloc(&h->Fpre, es * 3 * G * nc)) != cudaSuccess) {
                rc = fail(h, RT_ENOMEM, "cudaMalloc"); goto bad;
            }
        }
        h->q.capacity = nc;
        if ((e = cudaMallocHost((void **)&h->status_host, sizeof(unsigned))) != cudaSuccess) {
            rc = fail(h, RT_ENOMEM, "cudaMallocHost"); goto bad;
        }
        *h->status_host = 0;
        std::vector<double> tab((size_t)kHllNF * kHllNMU * 2);
        rtgb::hll_table(kHllNF, kHllNMU, tab.data());
        if ((e = cudaMemcpy(h->hll, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice)) != cudaSuccess) {
            rc = cuda_fail(h, e, "hll copy"); goto bad;
        }
        if (h->mixed) {
            std::vector<float> tabf(tab.begin(), tab.end());
            if ((rc = dalloc(h, &h->hllf, tabf.size()))) goto bad;
            if ((e = cudaMemcpy(h->hllf, tabf.data(), tabf.size() * sizeof(float), cudaMemcpyHostToDevice)) !=
                cudaSuccess) {
                rc = cuda_fail(h, e, "hll copy"); goto bad;
            }
        }
        if ((e = cudaMemset(h->q.counters, 0, kQueueCounters * sizeof(unsigned long long))) != cudaSuccess ||
            (e = cudaMemset(h->status, 0, sizeof(unsigned))) != cudaSuccess ||
            (e = cudaMemset(h->budget, 0, 4 * G * sizeof(double))) != cudaSuccess ||
            (e = cudaMemset(h->subcycles, 0, nc * sizeof(int32_t))) != cudaSuccess) {
            rc = cuda_fail(h, e, "cudaMemset"); goto bad;
        }
    }
    *out = h;
    return RT_OK;
bad:
    free_all(h);
    delete h;
    return rc;
}

void rt_destroy(rt_handle *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

int rt_set_stream(rt_handle *h, void *stream)
{
    if (!h) return RT_EINVAL;
    cudaStream_t s = stream ? (cudaStream_t)stream : h->own_stream;
    if (s != h->stream) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
        h->stream = s;
        invalidate_graph(h);
    }
    return RT_OK;
}

int rt_set_state(rt_handle *h, const double *nH, const double *xHII, const double *xHeII, const double *xHeIII,
                 const double *T, const double *N, const double *F, int device_ptrs)
{
    if (!h) return RT_EINVAL;
    if (!nH || !xHII || !xHeII || !xHeIII || !T || !N || !F) return fail(h, RT_EINVAL, "null state pointer");
    const long long nc = h->g.nc;
    const int G = h->G;
    if (!device_ptrs) {
        const StateView sv{nc, G, h->cr, nH, xHII, xHeII, xHeIII, T, N, F};
        long long bad = -1;
        switch (check_state(sv, &bad)) {
        case kStateGas: return fail(h, RT_EINVAL, "gas state out of range at cell " + std::to_string(bad));
        case kStatePhotons:
            return fail(h, RT_EINVAL, "photon state not finite / negative at cell " + std::to_string(bad));
        case kStateFlux: return fail(h, RT_EINVAL, "|F| > c_r N at cell " + std::to_string(bad));
        default: break;
        }
    }
    cudaMemcpyKind k = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    size_t b = (size_t)nc * sizeof(double);
    h->cur = 0;
    RT_CUDA(h, cudaMemcpyAsync(h->nH, nH, b, k, h->stream));
    RT_CUDA(h, cudaMemcpyAsync(h->xHII, xHII, b, k, h->stream));
    RT_CUDA(h, cudaMemcpyAsync(h->xHeII, xHeII, b, k, h->stream));
    RT_CUDA(h, cudaMemcpyAsync(h->xHeIII, xHeIII, b, k, h->stream));
    RT_CUDA(h, cudaMemcpyAsync(h->T, T, b, k, h->stream));
    if (!h->mixed) {
        RT_CUDA(h, cudaMemcpyAsync(h->N[0], N, G * b, k, h->stream));
        RT_CUDA(h, cudaMemcpyAsync(h->F[0], F, 3 * G * b, k, h->stream));
    } else if (device_ptrs) {
        cudaError_t ec = launch_convert_d2f((long long)G * nc, N, h->Nf[0], h->stream);
        if (ec == cudaSuccess) ec = launch_convert_d2f(3LL * G * nc, F, h->Ff[0], h->stream);
        if (ec != cudaSuccess) return cuda_fail(h, ec, "convert");
    } else {
        std::vector<float> nf(N, N + (size_t)G * nc), ff(F, F + (size_t)3 * G * nc);
        RT_CUDA(h, cudaMemcpyAsync(h->Nf[0], nf.data(), nf.size() * sizeof(float), cudaMemcpyHostToDevice,
                                   h->stream));
        RT_CUDA(h, cudaMemcpyAsync(h->Ff[0], ff.data(), ff.size() * sizeof(float), cudaMemcpyHostToDevice,
                                   h->stream));
        RT_CUDA(h, cudaStreamSynchronize(h->stream));
    }
    RT_CUDA(h, cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
    RT_CUDA(h, cudaMemsetAsync(h->q.counters, 0, kQueueCounters * sizeof(unsigned long long), h->stream));
    cudaError_t e = h->mixed ? launch_reduce_N_f32(G, nc, h->Nf[0], h->part, h->stream)
                             : launch_reduce_N(G, nc, h->N[0], h->part, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "reduce");
    e = launch_finalize_mode(G, 1, h->part, h->g.dx * h->g.dx * h->g.dx, nullptr, h->budget, h->q, h->status,
                             h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "finalize");
    if (!device_ptrs) RT_CUDA(h, cudaStreamSynchronize(h->stream));
    *h->status_host = 0;
    h->state_set = true;
    return RT_OK;
}

int rt_get_state(rt_handle *h, double *nH, double *xHII, double *xHeII, double *xHeIII, double *T, double *N,
                 double *F, int device_ptrs)
{
    if (!h) return RT_EINVAL;
    int rc = sync_and_check(h);
    cudaMemcpyKind k = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    size_t b = (size_t)h->g.nc * sizeof(double);
    if (nH) RT_CUDA(h, cudaMemcpyAsync(nH, h->nH, b, k, h->stream));
    if (xHII) RT_CUDA(h, cudaMemcpyAsync(xHII, h->xHII, b, k, h->stream));
    if (xHeII) RT_CUDA(h, cudaMemcpyAsync(xHeII, h->xHeII, b, k, h->stream));
    if (xHeIII) RT_CUDA(h, cudaMemcpyAsync(xHeIII, h->xHeIII, b, k, h->stream));
    if (T) RT_CUDA(h, cudaMemcpyAsync(T, h->T, b, k, h->stream));
    if (!h->mixed) {
        if (N) RT_CUDA(h, cudaMemcpyAsync(N, h->N[h->cur], h->G * b, k, h->stream));
        if (F) RT_CUDA(h, cudaMemcpyAsync(F, h->F[h->cur], 3 * h->G * b, k, h->stream));
    } else if (device_ptrs) {
        const long long n1 = (long long)h->G * h->g.nc;
        cudaError_t ec = cudaSuccess;
        if (N) ec = launch_convert_f2d(n1, h->Nf[h->cur], N, h->stream);
        if (F && ec == cudaSuccess) ec = launch_convert_f2d(3 * n1, h->Ff[h->cur], F, h->stream);
        if (ec != cudaSuccess) return cuda_fail(h, ec, "convert");
    } else {
        const size_t n1 = (size_t)h->G * h->g.nc;
        std::vector<float> tmp;
        if (N) {
            tmp.resize(n1);
            RT_CUDA(h, cudaMemcpyAsync(tmp.data(), h->Nf[h->cur], n1 * sizeof(float), cudaMemcpyDeviceToHost,
                                       h->stream));
            RT_CUDA(h, cudaStreamSynchronize(h->stream));
            for (size_t i = 0; i < n1; ++i) N[i] = tmp[i];
        }
        if (F) {
            tmp.resize(3 * n1);
            RT_CUDA(h, cudaMemcpyAsync(tmp.data(), h->Ff[h->cur], 3 * n1 * sizeof(float), cudaMemcpyDeviceToHost,
                                       h->stream));
            RT_CUDA(h, cudaStreamSynchronize(h->stream));
            for (size_t i = 0; i < 3 * n1; ++i) F[i] = tmp[i];
        }
    }
    if (!device_ptrs) RT_CUDA(h, cudaStreamSynchronize(h->stream));
    return rc;
}

int rt_set_sources(rt_handle *h, int n, const int32_t *ijk, const double *L)
{
    if (!h) return RT_EINVAL;
    if (n < 0 || (n > 0 && (!ijk || !L))) return fail(h, RT_EINVAL, "bad source arrays");
    const int G = h->G;
    std::map<long long, std::vector<double>> merged;
    std::vector<long long> order;
    std::vector<double> tot(G, 0.0);
    for (int s = 0; s < n; ++s) {
        int i = ijk[3 * s], j = ijk[3 * s + 1], k = ijk[3 * s + 2];
        if (i < 0 || j < 0 || k < 0 || i >= h->g.nx || j >= h->g.ny || k >= h->g.nz)
            return fail(h, RT_EINVAL, "source outside the grid");
        long long c = ((long long)k * h->g.ny + j) * h->g.nx + i;
        auto it = merged.find(c);
        if (it == merged.end()) {
            it = merged.emplace(c, std::vector<double>(G, 0.0)).first;
            order.push_back(c);
        }
        for (int g = 0; g < G; ++g) {
            double l = L[(size_t)s * G + g];
            if (!(l >= 0.0) || !std::isfinite(l)) return fail(h, RT_EINVAL, "bad source luminosity");
            it->second[g] += l;
            tot[g] += l;
        }
    }
    RT_CUDA(h, cudaStreamSynchronize(h->stream));
    if (h->src_cell) { cudaFree(h->src_cell); h->src_cell = nullptr; }
    if (h->src_L) { cudaFree(h->src_L); h->src_L = nullptr; }
    h->nsrc = 0;
    int m = (int)order.size();
    if (m > 0) {
        std::vector<double> Lh((size_t)m * G);
        for (int s = 0; s < m; ++s)
            for (int g = 0; g < G; ++g) Lh[(size_t)s * G + g] = merged[order[s]][g];
        int rc;
        if ((rc = dalloc(h, &h->src_cell, m)) || (rc = dalloc(h, &h->src_L, (size_t)m * G))) return rc;
        RT_CUDA(h, cudaMemcpy(h->src_cell, order.data(), m * sizeof(long long), cudaMemcpyHostToDevice));
        RT_CUDA(h, cudaMemcpy(h->src_L, Lh.data(), Lh.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    h->nsrc = m;
    h->src_Lsum_host = tot;
    if (h->src_cell_orig) { cudaFree(h->src_cell_orig); h->src_cell_orig = nullptr; }
    h->nsrc_orig = 0;
    if (n > 0) {
        std::vector<long long> oc(n);
        for (int s = 0; s < n; ++s)
            oc[s] = ((long long)ijk[3 * s + 2] * h->g.ny + ijk[3 * s + 1]) * h->g.nx + ijk[3 * s];
        int rc = dalloc(h, &h->src_cell_orig, n);
        if (rc) return rc;
        RT_CUDA(h, cudaMemcpy(h->src_cell_orig, oc.data(), n * sizeof(long long), cudaMemcpyHostToDevice));
    }
    h->nsrc_orig = n;
    invalidate_graph(h);
    return RT_OK;
}

int rt_set_inflow(rt_handle *h, int face, const double *state)
{
    if (!h) return RT_EINVAL;
    if (face < 0 || face > 5 || !state) return fail(h, RT_EINVAL, "bad inflow face or null state");
    if (h->g.bc[face] != RT_BC_INFLOW) return fail(h, RT_EINVAL, "face is not an RT_BC_INFLOW face");
    const int G = h->G;
    for (int g = 0; g < G; ++g) {
        const double *u = state + 4 * g;
        const double F2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
        const double cn = h->cr * u[0];
        if (!std::isfinite(u[0]) || !std::isfinite(F2) || !(u[0] >= 0.0) || F2 > cn * cn * (1.0 + 2e-8) + 1e-290)
            return fail(h, RT_EINVAL, "inflow state not realisable (needs N >= 0, |F| <= c_r N)");
    }
    RT_CUDA(h, cudaStreamSynchronize(h->stream));
    std::vector<double> buf((size_t)24 * G);
    RT_CUDA(h, cudaMemcpy(buf.data(), h->inflow_d, buf.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int g = 0; g < G; ++g)
        for (int k = 0; k < 4; ++k) buf[(size_t)24 * g + 4 * face + k] = state[4 * g + k];
    RT_CUDA(h, cudaMemcpy(h->inflow_d, buf.data(), buf.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (h->inflow_f) {
        std::vector<float> bf(buf.begin(), buf.end());
        RT_CUDA(h, cudaMemcpy(h->inflow_f, bf.data(), bf.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    invalidate_graph(h);
    return RT_OK;
}

int rt_set_scale_factor(rt_handle *h, double a)
{
    if (!h) return RT_EINVAL;
    if (!(a > 0.0) || !std::isfinite(a)) return fail(h, RT_EINVAL, "expansion factor must be > 0");
    if (!h->state_set) return fail(h, RT_EINVAL, "rt_set_state has not been called");
    const double r = h->opt.a_exp / a;
    if (r == 1.0) return RT_OK;
    const long long nc = h->g.nc;
    const int G = h->G;
    cudaError_t e;
    if (h->mixed) {
        e = launch_scale_f32((long long)G * nc, r * r * r, h->Nf[h->cur], h->stream);
        if (e == cudaSuccess) e = launch_scale_f32(3LL * G * nc, r * r * r * r, h->Ff[h->cur], h->stream);
    } else {
        e = launch_scale((long long)G * nc, r * r * r, h->N[h->cur], h->stream);
        if (e == cudaSuccess) e = launch_scale(3LL * G * nc, r * r * r * r, h->F[h->cur], h->stream);
    }
    if (e == cudaSuccess) e = launch_scale(nc, r * r * r, h->nH, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "scale");
    h->g.dx /= r;
    h->opt.a_exp = a;
    invalidate_graph(h);
    return RT_OK;
}

int rt_courant_dt(const rt_handle *h, double *dt)
{
    if (!h || !dt) return RT_EINVAL;
    *dt = courant(h);
    return RT_OK;
}

int rt_step(rt_handle *h, double dt)
{
    if (!h) return RT_EINVAL;
    int rc = check_dt(h, &dt);
    if (rc) return rc;
    return enqueue_step(h, dt);
}

int rt_run(rt_handle *h, double dt, int nsteps)
{
    if (!h) return RT_EINVAL;
    if (nsteps < 0) return fail(h, RT_EINVAL, "nsteps < 0");
    int rc = check_dt(h, &dt);
    if (rc) return rc;
    if (nsteps == 0) return RT_OK;
    // the graph holds two steps so that the ping-pong buffers line up again
    if (!h->graph || h->graph_dt != dt || h->graph_cur0 != h->cur) {
        invalidate_graph(h);
        cudaGraph_t graph;
        int cur0 = h->cur;
        RT_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        int r1 = enqueue_step(h, dt, true);
        int r2 = r1 ? r1 : enqueue_step(h, dt, true);
        cudaError_t ec = cudaStreamEndCapture(h->stream, &graph);
        h->cur = cur0;
        if (r2) return r2;
        if (ec != cudaSuccess) return cuda_fail(h, ec, "cudaStreamEndCapture");
        cudaError_t ei = cudaGraphInstantiate(&h->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) { h->graph = nullptr; return cuda_fail(h, ei, "cudaGraphInstantiate"); }
        h->graph_dt = dt;
        h->graph_cur0 = cur0;
    }
    int pairs = nsteps / 2;
    for (int k = 0; k < pairs; ++k) RT_CUDA(h, cudaGraphLaunch(h->graph, h->stream));
    if (nsteps % 2) return enqueue_step(h, dt);
    return RT_OK;
}

int rt_get_budget(rt_handle *h, double *out)
{
    if (!h || !out) return RT_EINVAL;
    int rc = sync_and_check(h);
    RT_CUDA(h, cudaMemcpy(out, h->budget, 4 * h->G * sizeof(double), cudaMemcpyDeviceToHost));
    return rc;
}

int rt_get_subcycles(rt_handle *h, int32_t *per_cell, int device_ptr)
{
    if (!h || !per_cell) return RT_EINVAL;
    int rc = sync_and_check(h);
    RT_CUDA(h, cudaMemcpy(per_cell, h->subcycles, h->g.nc * sizeof(int32_t),
                          device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    return rc;
}

int rt_set_thermo_routing(rt_handle *h, int pass1_attempts, int drain_budget, int drain2_budget,
                          long long drain2_min_cells)
{
    if (!h) return RT_EINVAL;
    ThermoParams d{};
    default_routing(d);
    h->routing.pass1_attempts = pass1_attempts > 0 ? pass1_attempts : d.pass1_attempts;
    h->routing.drain_budget = drain_budget > 0 ? drain_budget : d.drain_budget;
    h->routing.drain2_budget = drain2_budget > 0 ? drain2_budget : d.drain2_budget;
    h->routing.drain2_min = drain2_min_cells >= 0 ? drain2_min_cells : d.drain2_min;
    invalidate_graph(h);   // the captured launches carry the old routing
    return RT_OK;
}

int rt_set_profiling(rt_handle *h, int enable)
{
    if (!h) return RT_EINVAL;
    RT_CUDA(h, cudaStreamSynchronize(h->stream));
    prof_collect(h);
    h->prof = enable != 0;
    for (int k = 0; k < RT_NPHASES; ++k) { h->prof_ms[k] = 0.0; h->prof_n[k] = 0; }
    return RT_OK;
}

int rt_get_profile(rt_handle *h, double *ms, int64_t *launches)
{
    if (!h || !ms || !launches) return RT_EINVAL;
    int rc = sync_and_check(h);
    for (int k = 0; k < RT_NPHASES; ++k) { ms[k] = h->prof_ms[k]; launches[k] = h->prof_n[k]; }
    return rc;
}

int rt_step_vjp(rt_handle *h, double dt, double *lam_xHII, double *lam_xHeII, double *lam_xHeIII, double *lam_T,
                double *lam_N, double *lam_F, double *g_nH, double *g_L, long long *mismatches)
{
    if (!h) return RT_EINVAL;
    int rc = vjp_args(h, &dt, lam_xHII, lam_xHeII, lam_xHeIII, lam_T, lam_N, lam_F, g_nH, g_L);
    if (rc) return rc;
    const bool check = mismatches != nullptr;
    if ((rc = ensure_adj(h))) return rc;
    if (check) RT_CUDA(h, cudaMemsetAsync(h->adj_count, 0, sizeof(unsigned long long), h->stream));
    rc = enqueue_vjp(h, dt, lam_xHII, lam_xHeII, lam_xHeIII, lam_T, lam_N, lam_F, g_nH, g_L, check);
    if (rc) return rc;
    if (check) {
        rc = sync_and_check(h);
        if (rc) return rc;
        unsigned long long n = 0;
        RT_CUDA(h, cudaMemcpy(&n, h->adj_count, sizeof(n), cudaMemcpyDeviceToHost));
        *mismatches += (long long)n;
    }
    return RT_OK;
}

int rt_run_vjp(rt_handle *h, double dt, int nsteps, double *lam_xHII, double *lam_xHeII, double *lam_xHeIII,
               double *lam_T, double *lam_N, double *lam_F, double *g_nH, double *g_L, long long *mismatches)
{
    if (!h) return RT_EINVAL;
    if (nsteps < 0) return fail(h, RT_EINVAL, "nsteps < 0");
    int rc = vjp_args(h, &dt, lam_xHII, lam_xHeII, lam_xHeIII, lam_T, lam_N, lam_F, g_nH, g_L);
    if (rc) return rc;
    if (nsteps == 0) return RT_OK;
    const long long nc = h->g.nc;
    const size_t per = (size_t)(4 + 4 * h->G) * nc;   // gas x_HII, x_HeII, x_HeIII, T + N, F
    double *traj = nullptr;
    cudaError_t e = cudaMalloc((void **)&traj, per * nsteps * sizeof(double));
    if (e != cudaSuccess) return fail(h, RT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    auto copy_state = [&](double *dst, bool save) -> int {
        double *gas[4] = {h->xHII, h->xHeII, h->xHeIII, h->T};
        const size_t b1 = nc * sizeof(double);
        for (int k = 0; k < 4; ++k) {
            cudaError_t ee = save ? cudaMemcpyAsync(dst + k * nc, gas[k], b1, cudaMemcpyDeviceToDevice, h->stream)
                                  : cudaMemcpyAsync(gas[k], dst + k * nc, b1, cudaMemcpyDeviceToDevice, h->stream);
            if (ee != cudaSuccess) return cuda_fail(h, ee, "trajectory copy");
        }
        double *Nd = dst + 4 * nc, *Fd = Nd + (size_t)h->G * nc;
        const size_t bN = (size_t)h->G * nc * sizeof(double);
        cudaError_t e1 = save ? cudaMemcpyAsync(Nd, h->N[h->cur], bN, cudaMemcpyDeviceToDevice, h->stream)
                              : cudaMemcpyAsync(h->N[h->cur], Nd, bN, cudaMemcpyDeviceToDevice, h->stream);
        cudaError_t e2 = save ? cudaMemcpyAsync(Fd, h->F[h->cur], 3 * bN, cudaMemcpyDeviceToDevice, h->stream)
                              : cudaMemcpyAsync(h->F[h->cur], Fd, 3 * bN, cudaMemcpyDeviceToDevice, h->stream);
        if (e1 != cudaSuccess || e2 != cudaSuccess) return cuda_fail(h, e1 != cudaSuccess ? e1 : e2, "trajectory copy");
        return RT_OK;
    };
    const bool check = mismatches != nullptr;
    if ((rc = ensure_adj(h))) { cudaFree(traj); return rc; }
    if (check) RT_CUDA(h, cudaMemsetAsync(h->adj_count, 0, sizeof(unsigned long long), h->stream));
    invalidate_graph(h);
    // recompute the forward trajectory, keeping every step's input state
    for (int k = 0; k < nsteps && !rc; ++k) {
        rc = copy_state(traj + per * k, true);
        if (!rc) rc = enqueue_step(h, dt);
    }
    // reverse sweep; the handle ends at the state it started from
    for (int k = nsteps - 1; k >= 0 && !rc; --k) {
        rc = copy_state(traj + per * k, false);
        if (!rc) rc = enqueue_vjp(h, dt, lam_xHII, lam_xHeII, lam_xHeIII, lam_T, lam_N, lam_F, g_nH, g_L, check);
    }
    int rs = sync_and_check(h);
    cudaFree(traj);
    if (rc) return rc;
    if (rs) return rs;
    if (check) {
        unsigned long long n = 0;
        RT_CUDA(h, cudaMemcpy(&n, h->adj_count, sizeof(n), cudaMemcpyDeviceToHost));
        *mismatches += (long long)n;
    }
    return RT_OK;
}

int rt_sync(rt_handle *h)
{
    if (!h) return RT_EINVAL;
    return sync_and_check(h);
}

const char *rt_last_error(const rt_handle *h)
{
    if (!h) return kNoHandle;
    return h->err.c_str();
}

}  // extern "C"

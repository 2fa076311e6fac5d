// Batched RT steps over many independent boxes of uneven sizes (C-ABI
// rt_batch_*, declared in include/rt.h).
//
// Every box runs the same method as a single handle (paper Sec. 3:
// injection, transport, thermochemistry over the same dt): boxes share the
// cell width, the reduced light speed and the options, so one Courant step
// serves all of them; each box has its own size, boundary conditions, state,
// sources and number of photon groups.  Boxes with the same group count form
// a class whose cells are stored back to back ([G][cells of the class]
// photon arrays), so the thermochemistry of a whole class is one queue-
// balanced pass, and the transport of all boxes is one launch over a work
// list of (box, group, tile, z range) items of both tile shapes.  A step is
// captured as one CUDA graph by rt_batch_run.  rt_batch_autotune picks, per
// box side, the tile shape (32 x 8 or 16 x 16) and the planes per CTA that
// transport fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "rt_internal.h"

using namespace rtgb;

namespace {

constexpr int kRB = 256;

struct ClassData {
    int G = 0;
    long long nc = 0;
    GroupConsts gc{};
    double *nH = nullptr, *xHII = nullptr, *xHeII = nullptr, *xHeIII = nullptr, *T = nullptr;
    void *N[2] = {nullptr, nullptr};
    void *F[2] = {nullptr, nullptr};
    int32_t *sub = nullptr;
    Queue q{};
    unsigned *status = nullptr;    // shared status word (points into batch)
    // sources of the class: cell index within the class, luminosity [n][G]
    int nsrc = 0;
    long long *src_cell = nullptr;
    double *src_L = nullptr;
};

struct BoxHost {
    rt_grid grid;
    int G;
    int cls;
    long long cell_off;
    int shape = 0;        // transport tile shape (0: 32x8, 1: 16x16)
    int zc = 16;          // planes per CTA
    std::vector<int32_t> src_ijk;
    std::vector<double> src_L;
};

// one block per (box, group): sum N over the box's cells of that group
template <typename P>
__global__ void __launch_bounds__(kRB)
batch_reduce_kernel(const BatchBox *__restrict__ boxes, const int *__restrict__ bg_box, const int *__restrict__ bg_grp,
                    const void *const *__restrict__ Ncls, double *__restrict__ out, int k0)
{
    __shared__ double sh[kRB / 32];
    const int k = k0 + blockIdx.x;
    const BatchBox b = boxes[bg_box[k]];
    const P *N = reinterpret_cast<const P *>(Ncls[b.cls]) + (long long)bg_grp[k] * b.g.stride + b.cell_off;
    double acc = 0.0;
    for (long long i = threadIdx.x; i < b.g.nc; i += kRB) acc += (double)N[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kRB / 32; ++w) t += sh[w];
        out[k] = t;
    }
}

// per (box, group): fold the transport partials of its items (fixed order)
// and the photon sum into the cumulative budget [in_box, absorbed, outflow,
// emitted]; mode 1 (set_state) only sets in_box and clears the rest.
__global__ void batch_finalize_kernel(int k0, int nbg, int mode, const int *__restrict__ bg_item0,
                                      const int *__restrict__ bg_nitem, const int *__restrict__ bg_stride,
                                      const double *__restrict__ pin, const double *__restrict__ pout,
                                      const double *__restrict__ red, const double *__restrict__ emitted, double V,
                                      double *__restrict__ budget, unsigned *status)
{
    for (int k = k0 + blockIdx.x * blockDim.x + threadIdx.x; k < k0 + nbg; k += gridDim.x * blockDim.x) {
        double C = red[k];
        double *b = budget + 4 * (long long)k;
        b[0] = C * V;
        if (mode == 0) {
            double A = 0.0, B = 0.0;
            for (int i = 0; i < bg_nitem[k]; ++i) {
                int it = bg_item0[k] + i * bg_stride[k];
                A += pin[it];
                B += pout[it];
            }
            b[1] += (A - C) * V;
            b[2] += B;
            b[3] += emitted[k];
            if (!isfinite(A) || !isfinite(B) || !isfinite(C)) atomicOr(status, kStatusNonFinite);
        } else {
            b[1] = b[2] = b[3] = 0.0;
        }
    }
}

__global__ void reset_counters_kernel(unsigned long long *c, int n)
{
    if (threadIdx.x < n) c[threadIdx.x] = 0ULL;
}

}  // namespace

struct rt_batch {
    int nbox = 0;
    double dx = 0.0, cr = 0.0;
    rt_options opt{};
    bool mixed = false;
    int device = 0, n_sm = 1;
    cudaStream_t own_stream = nullptr, stream = nullptr;
    std::vector<BoxHost> box;
    std::vector<ClassData> cls;
    int cur = 0;
    // device tables
    BatchBox *d_boxes = nullptr;
    BatchItem *d_items = nullptr;
    int n_items = 0, n_items_shape0 = 0;
    void **d_Ncls[2] = {nullptr, nullptr};   // per ping-pong side: class base pointers
    void **d_Fcls[2] = {nullptr, nullptr};
    double *d_pin = nullptr, *d_pout = nullptr;
    int nbg = 0;
    int *d_bg_box = nullptr, *d_bg_grp = nullptr, *d_bg_item0 = nullptr, *d_bg_nitem = nullptr, *d_bg_stride = nullptr;
    std::vector<int> bg_first;      // first box-group index of each box
    double *d_red = nullptr, *d_budget = nullptr, *d_emitted = nullptr;
    double *hll = nullptr;
    float *hllf = nullptr;
    unsigned *status = nullptr;
    unsigned *status_host = nullptr;
    bool state_set = false;
    cudaGraphExec_t graph = nullptr;
    double graph_dt = 0.0;
    int graph_cur0 = 0;
    double emitted_dt = -1.0;
    std::string err;
};

namespace {

int bfail(rt_batch *b, int code, const std::string &m)
{
    if (b) b->err = m;
    return code;
}

int bcuda(rt_batch *b, cudaError_t e, const char *what)
{
    return bfail(b, RT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define B_CUDA(b, call)                                       \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return bcuda(b, e_, #call);    \
    } while (0)

template <typename T>
int balloc(rt_batch *b, T **p, size_t n)
{
    cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return bfail(b, RT_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return RT_OK;
}

void bfree_all(rt_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (ClassData &c : b->cls) {
        void *ptrs[] = {c.nH, c.xHII, c.xHeII, c.xHeIII, c.T, c.N[0], c.N[1], c.F[0], c.F[1], c.sub,
                        c.q.a.cell, c.q.a.t_left, c.q.a.dt_tc, c.q.a.attempts, c.q.b.cell, c.q.b.t_left,
                        c.q.b.dt_tc, c.q.b.attempts, c.q.counters, c.q.fscale, c.src_cell, c.src_L};
        for (void *p : ptrs)
            if (p) cudaFree(p);
    }
    void *ptrs[] = {b->d_boxes, b->d_items, b->d_Ncls[0], b->d_Ncls[1], b->d_Fcls[0], b->d_Fcls[1], b->d_pin,
                    b->d_pout, b->d_bg_box, b->d_bg_grp, b->d_bg_item0, b->d_bg_nitem, b->d_bg_stride, b->d_red,
                    b->d_budget, b->d_emitted, b->hll, b->hllf, b->status};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (b->status_host) cudaFreeHost(b->status_host);
    if (b->own_stream) cudaStreamDestroy(b->own_stream);
}

GridDev box_griddev(const BoxHost &bx, const ClassData &c)
{
    GridDev g{};
    g.nx = bx.grid.nx;
    g.ny = bx.grid.ny;
    g.nz = bx.grid.nz;
    g.nc = (long long)g.nx * g.ny * g.nz;
    g.stride = c.nc;
    g.dx = bx.grid.dx_cm;
    for (int i = 0; i < 6; ++i) g.bc[i] = bx.grid.bc[i];
    return g;
}

// Work list: shape-0 boxes first, then shape-1 boxes; per box, groups,
// then (z chunk, y tile, x tile).  Also the (box, group) item ranges.
int build_items(rt_batch *b)
{
    std::vector<BatchItem> items;
    std::vector<int> bg_item0(b->nbg), bg_nitem(b->nbg), bg_stride(b->nbg, 1);
    for (int shape = 0; shape < 2; ++shape) {
        const int TX = shape == 0 ? 32 : 16, TY = shape == 0 ? 8 : 16;
        for (int i = 0; i < b->nbox; ++i) {
            const BoxHost &bx = b->box[i];
            if (bx.shape != shape) continue;
            const int nx = bx.grid.nx, ny = bx.grid.ny, nz = bx.grid.nz;
            for (int gg = 0; gg < bx.G; ++gg) {
                int k = b->bg_first[i] + gg;
                bg_item0[k] = (int)items.size();
                int n = 0;
                for (int z0 = 0; z0 < nz; z0 += bx.zc)
                    for (int y0 = 0; y0 < ny; y0 += TY)
                        for (int x0 = 0; x0 < nx; x0 += TX) {
                            items.push_back(BatchItem{i, gg, x0, y0, z0, std::min(z0 + bx.zc, nz)});
                            ++n;
                        }
                bg_nitem[k] = n;
            }
        }
        if (shape == 0) b->n_items_shape0 = (int)items.size();
    }
    b->n_items = (int)items.size();
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_pin) cudaFree(b->d_pin);
    if (b->d_pout) cudaFree(b->d_pout);
    b->d_items = nullptr;
    b->d_pin = b->d_pout = nullptr;
    int rc;
    if ((rc = balloc(b, &b->d_items, items.size())) || (rc = balloc(b, &b->d_pin, items.size())) ||
        (rc = balloc(b, &b->d_pout, items.size())))
        return rc;
    B_CUDA(b, cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
    B_CUDA(b, cudaMemcpy(b->d_bg_item0, bg_item0.data(), b->nbg * sizeof(int), cudaMemcpyHostToDevice));
    B_CUDA(b, cudaMemcpy(b->d_bg_nitem, bg_nitem.data(), b->nbg * sizeof(int), cudaMemcpyHostToDevice));
    B_CUDA(b, cudaMemcpy(b->d_bg_stride, bg_stride.data(), b->nbg * sizeof(int), cudaMemcpyHostToDevice));
    return RT_OK;
}

ThermoParams class_params(const rt_batch *b, const ClassData &c, double dt)
{
    ThermoParams p{};
    p.nc = c.nc;
    p.dt = dt;
    p.cr = b->cr;
    p.X = b->opt.X;
    double Y = 1.0 - b->opt.X;
    p.he_ratio = (Y > 0.0) ? Y / (4.0 * b->opt.X) : 0.0;
    p.kfac = (5.0 / 3.0 - 1.0) * b->opt.X / 1.380649e-16;
    p.a_exp = b->opt.a_exp;
    p.isothermal = b->opt.isothermal ? 1 : 0;
    p.helium = (Y > 0.0) ? 1 : 0;
    p.case_b = 1;
    p.max_sub = b->opt.max_subcycles;
    default_routing(p);
    p.gc = c.gc;
    derive_group_terms(p);
    return p;
}

int upload_emitted(rt_batch *b, double dt)
{
    std::vector<double> em(b->nbg, 0.0);
    for (int i = 0; i < b->nbox; ++i) {
        const BoxHost &bx = b->box[i];
        int ns = (int)bx.src_ijk.size() / 3;
        for (int s = 0; s < ns; ++s)
            for (int g = 0; g < bx.G; ++g) em[b->bg_first[i] + g] += bx.src_L[(size_t)s * bx.G + g] * dt;
    }
    B_CUDA(b, cudaMemcpy(b->d_emitted, em.data(), em.size() * sizeof(double), cudaMemcpyHostToDevice));
    b->emitted_dt = dt;
    return RT_OK;
}

int enqueue_batch_step(rt_batch *b, double dt)
{
    const double V = b->dx * b->dx * b->dx;
    const bool f32 = b->mixed;
    cudaError_t e;
    for (ClassData &c : b->cls) {
        if (c.nsrc <= 0) continue;
        if (f32) e = launch_inject_f32(c.nsrc, c.G, c.nc, c.src_cell, c.src_L, dt / V, (float *)c.N[b->cur], b->stream);
        else e = launch_inject(c.nsrc, c.G, c.nc, c.src_cell, c.src_L, dt / V, (double *)c.N[b->cur], b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "inject");
    }
    const int nxt = 1 - b->cur;
    const void *tab = f32 ? (const void *)b->hllf : (const void *)b->hll;
    e = launch_transport_batch_all(b->d_items, b->d_boxes, b->n_items_shape0, b->n_items, f32, b->opt.flux, b->cr,
                                   dt, b->dx, (const void *const *)b->d_Ncls[b->cur],
                                   (const void *const *)b->d_Fcls[b->cur], b->d_Ncls[nxt], b->d_Fcls[nxt], tab,
                                   b->d_pin, b->d_pout, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "transport");
    b->cur = nxt;
    for (ClassData &c : b->cls) {
        ThermoParams tp = class_params(b, c, dt);
        if (f32)
            e = launch_thermo_mixed(tp, c.G, b->opt.precision == RT_MIXED32, c.nH, c.xHII, c.xHeII, c.xHeIII, c.T,
                                    (float *)c.N[b->cur], (float *)c.F[b->cur], nullptr, nullptr, c.sub, c.q,
                                    b->status, b->n_sm, b->stream);
        else
            e = launch_thermo(tp, c.G, c.nH, c.xHII, c.xHeII, c.xHeIII, c.T, (double *)c.N[b->cur],
                              (double *)c.F[b->cur], nullptr, nullptr, c.sub, c.q, b->status, b->n_sm, b->stream);
        if (e != cudaSuccess) return bcuda(b, e, "thermo");
        reset_counters_kernel<<<1, 32, 0, b->stream>>>(c.q.counters, kQueueCounters);
    }
    if (f32)
        batch_reduce_kernel<float><<<b->nbg, kRB, 0, b->stream>>>(b->d_boxes, b->d_bg_box, b->d_bg_grp,
                                                                  (const void *const *)b->d_Ncls[b->cur], b->d_red, 0);
    else
        batch_reduce_kernel<double><<<b->nbg, kRB, 0, b->stream>>>(b->d_boxes, b->d_bg_box, b->d_bg_grp,
                                                                   (const void *const *)b->d_Ncls[b->cur], b->d_red, 0);
    batch_finalize_kernel<<<(b->nbg + 255) / 256, 256, 0, b->stream>>>(0, b->nbg, 0, b->d_bg_item0, b->d_bg_nitem,
                                                                       b->d_bg_stride, b->d_pin, b->d_pout, b->d_red,
                                                                       b->d_emitted, V, b->d_budget, b->status);
    e = cudaMemcpyAsync(b->status_host, b->status, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "status copy");
    return RT_OK;
}

int bstatus_code(rt_batch *b, unsigned st)
{
    if (st & kStatusNonFinite) return bfail(b, RT_ENONFINITE, "non-finite value in the state");
    if (st & kStatusSubcycle) return bfail(b, RT_ESUBCYCLE, "a cell exceeded max_subcycles");
    if (st & kStatusQueue) return bfail(b, RT_EQUEUE, "work queue overflow");
    return RT_OK;
}

int bsync(rt_batch *b)
{
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    unsigned st = 0;
    B_CUDA(b, cudaMemcpy(&st, b->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    return bstatus_code(b, st);
}

int bcheck_dt(rt_batch *b, double *dt)
{
    if (!b->state_set) return bfail(b, RT_EINVAL, "no box state has been set");
    double dc = b->opt.cfl * b->dx / (3.0 * b->cr);
    if (!(*dt > 0.0)) *dt = dc;
    if (!std::isfinite(*dt)) return bfail(b, RT_EINVAL, "dt is not finite");
    if (*dt > dc * (1.0 + 1e-12)) return bfail(b, RT_EDT, "dt above the Courant limit CFL dx/(3 c_r)");
    unsigned st = *(volatile unsigned *)b->status_host;
    if (st) return bstatus_code(b, st);
    if (b->emitted_dt != *dt) {
        int rc = upload_emitted(b, *dt);
        if (rc) return rc;
    }
    return RT_OK;
}

int upload_sources(rt_batch *b)
{
    for (size_t k = 0; k < b->cls.size(); ++k) {
        ClassData &c = b->cls[k];
        std::map<long long, std::vector<double>> merged;
        std::vector<long long> order;
        for (int i = 0; i < b->nbox; ++i) {
            const BoxHost &bx = b->box[i];
            if (bx.cls != (int)k) continue;
            int ns = (int)bx.src_ijk.size() / 3;
            for (int s = 0; s < ns; ++s) {
                long long cell = bx.cell_off + ((long long)bx.src_ijk[3 * s + 2] * bx.grid.ny + bx.src_ijk[3 * s + 1]) *
                                                   bx.grid.nx + bx.src_ijk[3 * s];
                auto it = merged.find(cell);
                if (it == merged.end()) {
                    it = merged.emplace(cell, std::vector<double>(c.G, 0.0)).first;
                    order.push_back(cell);
                }
                for (int g = 0; g < c.G; ++g) it->second[g] += bx.src_L[(size_t)s * c.G + g];
            }
        }
        if (c.src_cell) { cudaFree(c.src_cell); c.src_cell = nullptr; }
        if (c.src_L) { cudaFree(c.src_L); c.src_L = nullptr; }
        c.nsrc = (int)order.size();
        if (c.nsrc) {
            std::vector<double> Lh((size_t)c.nsrc * c.G);
            for (int s = 0; s < c.nsrc; ++s)
                for (int g = 0; g < c.G; ++g) Lh[(size_t)s * c.G + g] = merged[order[s]][g];
            int rc;
            if ((rc = balloc(b, &c.src_cell, c.nsrc)) || (rc = balloc(b, &c.src_L, Lh.size()))) return rc;
            B_CUDA(b, cudaMemcpy(c.src_cell, order.data(), c.nsrc * sizeof(long long), cudaMemcpyHostToDevice));
            B_CUDA(b, cudaMemcpy(c.src_L, Lh.data(), Lh.size() * sizeof(double), cudaMemcpyHostToDevice));
        }
    }
    b->emitted_dt = -1.0;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    return RT_OK;
}

}  // namespace

extern "C" {

int rt_batch_create(int n_boxes, const rt_grid *grids, const int *n_groups, const rt_options *opt, double c_r,
                    const double *const *sigN, const double *const *sigE, const double *const *egy, rt_batch **out)
{
    if (!out) return RT_EINVAL;
    *out = nullptr;
    if (n_boxes < 1 || !grids || !n_groups || !opt || !sigN || !sigE || !egy) return RT_EINVAL;
    if (!(c_r > 0.0) || !std::isfinite(c_r)) return RT_EINVAL;
    if (!(opt->X > 0.0 && opt->X <= 1.0) || !(opt->cfl > 0.0 && opt->cfl <= 1.0)) return RT_EINVAL;
    if ((opt->flux != RT_GLF && opt->flux != RT_HLL) || opt->otsa != 1 || opt->smooth != 0) return RT_EINVAL;
    if (opt->precision != RT_FP64 && opt->precision != RT_MIXED && opt->precision != RT_MIXED32) return RT_EINVAL;
    if (!(opt->a_exp > 0.0) || opt->max_subcycles < 1) return RT_EINVAL;
    const double dx = grids[0].dx_cm;
    long long total = 0;
    std::map<int, int> cls_of_G;
    for (int i = 0; i < n_boxes; ++i) {
        const rt_grid &g = grids[i];
        if (g.nx < 1 || g.ny < 1 || g.nz < 1 || g.dx_cm != dx || !(dx > 0.0)) return RT_EINVAL;
        for (int k = 0; k < 6; ++k)
            if (g.bc[k] < RT_BC_OUTFLOW || g.bc[k] > RT_BC_PERIODIC) return RT_EINVAL;
        for (int d = 0; d < 3; ++d)
            if ((g.bc[2 * d] == RT_BC_PERIODIC) != (g.bc[2 * d + 1] == RT_BC_PERIODIC)) return RT_EINVAL;
        if (n_groups[i] < 1 || n_groups[i] > RT_MAX_GROUPS || !sigN[i] || !sigE[i] || !egy[i]) return RT_EINVAL;
        total += (long long)g.nx * g.ny * g.nz;
    }
    if (total >= (1LL << 31)) return RT_EINVAL;
    rt_batch *b = new rt_batch();
    b->nbox = n_boxes;
    b->dx = dx;
    b->cr = c_r;
    b->opt = *opt;
    b->mixed = opt->precision != RT_FP64;
    // classes by group count, constants from the first box of each class
    for (int i = 0; i < n_boxes; ++i) {
        int G = n_groups[i];
        if (!cls_of_G.count(G)) {
            cls_of_G[G] = (int)b->cls.size();
            ClassData c;
            c.G = G;
            for (int g = 0; g < G; ++g) {
                for (int j = 0; j < 3; ++j) {
                    c.gc.sigN[g][j] = sigN[i][3 * g + j];
                    c.gc.sigE[g][j] = sigE[i][3 * g + j];
                }
                c.gc.egy[g] = egy[i][g];
            }
            b->cls.push_back(c);
        }
        const ClassData &c = b->cls[cls_of_G[G]];
        for (int g = 0; g < G; ++g) {   // boxes of a class must share its constants
            for (int j = 0; j < 3; ++j)
                if (c.gc.sigN[g][j] != sigN[i][3 * g + j] || c.gc.sigE[g][j] != sigE[i][3 * g + j]) {
                    delete b;
                    return RT_EINVAL;
                }
            if (c.gc.egy[g] != egy[i][g] || !(egy[i][g] > 0.0)) { delete b; return RT_EINVAL; }
        }
        BoxHost bx;
        bx.grid = grids[i];
        bx.G = G;
        bx.cls = cls_of_G[G];
        bx.cell_off = b->cls[bx.cls].nc;
        b->cls[bx.cls].nc += (long long)grids[i].nx * grids[i].ny * grids[i].nz;
        int side = std::min(grids[i].nx, grids[i].ny);
        bx.shape = (side % 32 == 0) ? 0 : 1;
        bx.zc = 16;
        b->box.push_back(bx);
    }
    int rc = RT_OK;
    cudaError_t e;
    if ((e = cudaGetDevice(&b->device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&b->n_sm, cudaDevAttrMultiProcessorCount, b->device)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->own_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        rc = bcuda(b, e, "setup");
        goto bad;
    }
    b->stream = b->own_stream;
    transport_init();
    {
        const size_t pb = b->mixed ? sizeof(float) : sizeof(double);
        for (ClassData &c : b->cls) {
            const size_t nc = (size_t)c.nc, G = (size_t)c.G;
            if ((rc = balloc(b, &c.nH, nc)) || (rc = balloc(b, &c.xHII, nc)) || (rc = balloc(b, &c.xHeII, nc)) ||
                (rc = balloc(b, &c.xHeIII, nc)) || (rc = balloc(b, &c.T, nc)) || (rc = balloc(b, &c.sub, nc)) ||
                (rc = balloc(b, &c.q.a.cell, nc)) || (rc = balloc(b, &c.q.a.t_left, nc)) ||
                (rc = balloc(b, &c.q.a.dt_tc, nc)) || (rc = balloc(b, &c.q.a.attempts, nc)) ||
                (rc = balloc(b, &c.q.b.cell, nc)) || (rc = balloc(b, &c.q.b.t_left, nc)) ||
                (rc = balloc(b, &c.q.b.dt_tc, nc)) || (rc = balloc(b, &c.q.b.attempts, nc)) ||
                (rc = balloc(b, &c.q.counters, kQueueCounters)) || (rc = balloc(b, &c.q.fscale, G * nc)))
                goto bad;
            c.q.capacity = c.nc;
            for (int k = 0; k < 2; ++k) {
                if ((e = cudaMalloc(&c.N[k], G * nc * pb)) != cudaSuccess ||
                    (e = cudaMalloc(&c.F[k], 3 * G * nc * pb)) != cudaSuccess) {
                    rc = bfail(b, RT_ENOMEM, "cudaMalloc");
                    goto bad;
                }
                cudaMemset(c.N[k], 0, G * nc * pb);
                cudaMemset(c.F[k], 0, 3 * G * nc * pb);
            }
            cudaMemset(c.q.counters, 0, kQueueCounters * sizeof(unsigned long long));
            cudaMemset(c.sub, 0, nc * sizeof(int32_t));
        }
        // box descriptors and (box, group) tables
        std::vector<BatchBox> hb(n_boxes);
        std::vector<int> bg_box, bg_grp;
        for (int i = 0; i < n_boxes; ++i) {
            hb[i].g = box_griddev(b->box[i], b->cls[b->box[i].cls]);
            hb[i].cell_off = b->box[i].cell_off;
            hb[i].cls = b->box[i].cls;
            hb[i].G = b->box[i].G;
            b->bg_first.push_back((int)bg_box.size());
            for (int g = 0; g < b->box[i].G; ++g) {
                bg_box.push_back(i);
                bg_grp.push_back(g);
            }
        }
        b->nbg = (int)bg_box.size();
        const int ncls = (int)b->cls.size();
        if ((rc = balloc(b, &b->d_boxes, n_boxes)) || (rc = balloc(b, &b->d_bg_box, b->nbg)) ||
            (rc = balloc(b, &b->d_bg_grp, b->nbg)) || (rc = balloc(b, &b->d_bg_item0, b->nbg)) ||
            (rc = balloc(b, &b->d_bg_nitem, b->nbg)) || (rc = balloc(b, &b->d_bg_stride, b->nbg)) ||
            (rc = balloc(b, &b->d_red, b->nbg)) || (rc = balloc(b, &b->d_budget, 4 * (size_t)b->nbg)) ||
            (rc = balloc(b, &b->d_emitted, b->nbg)) || (rc = balloc(b, &b->status, 1)) ||
            (rc = balloc(b, &b->hll, (size_t)kHllNF * kHllNMU * 2)) || (rc = balloc(b, &b->d_Ncls[0], ncls)) ||
            (rc = balloc(b, &b->d_Ncls[1], ncls)) || (rc = balloc(b, &b->d_Fcls[0], ncls)) ||
            (rc = balloc(b, &b->d_Fcls[1], ncls)))
            goto bad;
        cudaMemcpy(b->d_boxes, hb.data(), n_boxes * sizeof(BatchBox), cudaMemcpyHostToDevice);
        cudaMemcpy(b->d_bg_box, bg_box.data(), b->nbg * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(b->d_bg_grp, bg_grp.data(), b->nbg * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemset(b->d_budget, 0, 4 * (size_t)b->nbg * sizeof(double));
        cudaMemset(b->status, 0, sizeof(unsigned));
        for (int k = 0; k < 2; ++k) {
            std::vector<void *> np(ncls), fp(ncls);
            for (int j = 0; j < ncls; ++j) {
                np[j] = b->cls[j].N[k];
                fp[j] = b->cls[j].F[k];
            }
            cudaMemcpy(b->d_Ncls[k], np.data(), ncls * sizeof(void *), cudaMemcpyHostToDevice);
            cudaMemcpy(b->d_Fcls[k], fp.data(), ncls * sizeof(void *), cudaMemcpyHostToDevice);
        }
        std::vector<double> tab((size_t)kHllNF * kHllNMU * 2);
        rtgb::hll_table(kHllNF, kHllNMU, tab.data());
        cudaMemcpy(b->hll, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (b->mixed) {
            std::vector<float> tf(tab.begin(), tab.end());
            if ((rc = balloc(b, &b->hllf, tf.size()))) goto bad;
            cudaMemcpy(b->hllf, tf.data(), tf.size() * sizeof(float), cudaMemcpyHostToDevice);
        }
        if ((e = cudaMallocHost((void **)&b->status_host, sizeof(unsigned))) != cudaSuccess) {
            rc = bfail(b, RT_ENOMEM, "cudaMallocHost");
            goto bad;
        }
        *b->status_host = 0;
        if ((rc = build_items(b))) goto bad;
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) { rc = bcuda(b, e, "setup"); goto bad; }
    }
    *out = b;
    return RT_OK;
bad:
    bfree_all(b);
    delete b;
    return rc;
}

void rt_batch_destroy(rt_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    bfree_all(b);
    delete b;
}

int rt_batch_set_stream(rt_batch *b, void *stream)
{
    if (!b) return RT_EINVAL;
    cudaStream_t s = stream ? (cudaStream_t)stream : b->own_stream;
    if (s != b->stream) {
        B_CUDA(b, cudaStreamSynchronize(b->stream));
        b->stream = s;
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    }
    return RT_OK;
}

int rt_batch_set_box_state(rt_batch *b, int box, const double *nH, const double *xHII, const double *xHeII,
                           const double *xHeIII, const double *T, const double *N, const double *F, int device_ptrs)
{
    if (!b) return RT_EINVAL;
    if (box < 0 || box >= b->nbox) return bfail(b, RT_EINVAL, "box index out of range");
    if (!nH || !xHII || !xHeII || !xHeIII || !T || !N || !F) return bfail(b, RT_EINVAL, "null state pointer");
    const BoxHost &bx = b->box[box];
    ClassData &c = b->cls[bx.cls];
    const long long nc = (long long)bx.grid.nx * bx.grid.ny * bx.grid.nz;
    const int G = bx.G;
    if (!device_ptrs) {
        for (long long i = 0; i < nc; ++i) {
            bool ok = std::isfinite(nH[i]) && nH[i] > 0.0 && xHII[i] >= 1e-6 && xHII[i] <= 1.0 && xHeII[i] >= 0.0 &&
                      xHeIII[i] >= 0.0 && xHeII[i] + xHeIII[i] <= 1.0 && std::isfinite(T[i]) && T[i] > 0.0;
            if (!ok) return bfail(b, RT_EINVAL, "gas state out of range");
            for (int g = 0; g < G; ++g) {
                double n = N[(size_t)g * nc + i];
                if (!(std::isfinite(n) && n >= 0.0)) return bfail(b, RT_EINVAL, "photon state out of range");
            }
        }
    }
    cudaMemcpyKind k = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t bytes = (size_t)nc * sizeof(double);
    const long long off = bx.cell_off;
    B_CUDA(b, cudaMemcpyAsync(c.nH + off, nH, bytes, k, b->stream));
    B_CUDA(b, cudaMemcpyAsync(c.xHII + off, xHII, bytes, k, b->stream));
    B_CUDA(b, cudaMemcpyAsync(c.xHeII + off, xHeII, bytes, k, b->stream));
    B_CUDA(b, cudaMemcpyAsync(c.xHeIII + off, xHeIII, bytes, k, b->stream));
    B_CUDA(b, cudaMemcpyAsync(c.T + off, T, bytes, k, b->stream));
    for (int g = 0; g < G; ++g) {
        for (int comp = -1; comp < 3; ++comp) {
            const double *src = comp < 0 ? N + (size_t)g * nc : F + ((size_t)3 * g + comp) * nc;
            long long dst_off = comp < 0 ? (long long)g * c.nc + off : (3LL * g + comp) * c.nc + off;
            if (!b->mixed) {
                double *dst = (double *)(comp < 0 ? c.N[b->cur] : c.F[b->cur]) + dst_off;
                B_CUDA(b, cudaMemcpyAsync(dst, src, bytes, k, b->stream));
            } else {
                float *dst = (float *)(comp < 0 ? c.N[b->cur] : c.F[b->cur]) + dst_off;
                if (device_ptrs) {
                    cudaError_t e = launch_convert_d2f(nc, src, dst, b->stream);
                    if (e != cudaSuccess) return bcuda(b, e, "convert");
                } else {
                    std::vector<float> tmp(src, src + nc);
                    B_CUDA(b, cudaMemcpyAsync(dst, tmp.data(), nc * sizeof(float), cudaMemcpyHostToDevice, b->stream));
                    B_CUDA(b, cudaStreamSynchronize(b->stream));
                }
            }
        }
    }
    if (!device_ptrs) B_CUDA(b, cudaStreamSynchronize(b->stream));
    b->state_set = true;
    // the budget of this box restarts from its new photon content
    const int k0 = b->bg_first[box];
    if (b->mixed)
        batch_reduce_kernel<float><<<G, kRB, 0, b->stream>>>(b->d_boxes, b->d_bg_box, b->d_bg_grp,
                                                             (const void *const *)b->d_Ncls[b->cur], b->d_red, k0);
    else
        batch_reduce_kernel<double><<<G, kRB, 0, b->stream>>>(b->d_boxes, b->d_bg_box, b->d_bg_grp,
                                                              (const void *const *)b->d_Ncls[b->cur], b->d_red, k0);
    batch_finalize_kernel<<<1, 32, 0, b->stream>>>(k0, G, 1, b->d_bg_item0, b->d_bg_nitem, b->d_bg_stride, b->d_pin,
                                                   b->d_pout, b->d_red, b->d_emitted, b->dx * b->dx * b->dx,
                                                   b->d_budget, b->status);
    B_CUDA(b, cudaMemsetAsync(b->status, 0, sizeof(unsigned), b->stream));
    *b->status_host = 0;
    B_CUDA(b, cudaGetLastError());
    return RT_OK;
}

int rt_batch_get_box_state(rt_batch *b, int box, double *nH, double *xHII, double *xHeII, double *xHeIII, double *T,
                           double *N, double *F, int device_ptrs)
{
    if (!b) return RT_EINVAL;
    if (box < 0 || box >= b->nbox) return bfail(b, RT_EINVAL, "box index out of range");
    int rc = bsync(b);
    const BoxHost &bx = b->box[box];
    ClassData &c = b->cls[bx.cls];
    const long long nc = (long long)bx.grid.nx * bx.grid.ny * bx.grid.nz;
    cudaMemcpyKind k = device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t bytes = (size_t)nc * sizeof(double);
    const long long off = bx.cell_off;
    if (nH) B_CUDA(b, cudaMemcpyAsync(nH, c.nH + off, bytes, k, b->stream));
    if (xHII) B_CUDA(b, cudaMemcpyAsync(xHII, c.xHII + off, bytes, k, b->stream));
    if (xHeII) B_CUDA(b, cudaMemcpyAsync(xHeII, c.xHeII + off, bytes, k, b->stream));
    if (xHeIII) B_CUDA(b, cudaMemcpyAsync(xHeIII, c.xHeIII + off, bytes, k, b->stream));
    if (T) B_CUDA(b, cudaMemcpyAsync(T, c.T + off, bytes, k, b->stream));
    for (int g = 0; g < bx.G; ++g) {
        for (int comp = -1; comp < 3; ++comp) {
            double *dst = comp < 0 ? (N ? N + (size_t)g * nc : nullptr) : (F ? F + ((size_t)3 * g + comp) * nc : nullptr);
            if (!dst) continue;
            long long src_off = comp < 0 ? (long long)g * c.nc + off : (3LL * g + comp) * c.nc + off;
            if (!b->mixed) {
                const double *src = (const double *)(comp < 0 ? c.N[b->cur] : c.F[b->cur]) + src_off;
                B_CUDA(b, cudaMemcpyAsync(dst, src, bytes, k, b->stream));
            } else {
                const float *src = (const float *)(comp < 0 ? c.N[b->cur] : c.F[b->cur]) + src_off;
                if (device_ptrs) {
                    cudaError_t e = launch_convert_f2d(nc, src, dst, b->stream);
                    if (e != cudaSuccess) return bcuda(b, e, "convert");
                } else {
                    std::vector<float> tmp(nc);
                    B_CUDA(b, cudaMemcpyAsync(tmp.data(), src, nc * sizeof(float), cudaMemcpyDeviceToHost, b->stream));
                    B_CUDA(b, cudaStreamSynchronize(b->stream));
                    for (long long i = 0; i < nc; ++i) dst[i] = tmp[i];
                }
            }
        }
    }
    if (!device_ptrs) B_CUDA(b, cudaStreamSynchronize(b->stream));
    return rc;
}

int rt_batch_set_box_sources(rt_batch *b, int box, int n, const int32_t *ijk, const double *L)
{
    if (!b) return RT_EINVAL;
    if (box < 0 || box >= b->nbox) return bfail(b, RT_EINVAL, "box index out of range");
    if (n < 0 || (n > 0 && (!ijk || !L))) return bfail(b, RT_EINVAL, "bad source arrays");
    BoxHost &bx = b->box[box];
    for (int s = 0; s < n; ++s) {
        if (ijk[3 * s] < 0 || ijk[3 * s + 1] < 0 || ijk[3 * s + 2] < 0 || ijk[3 * s] >= bx.grid.nx ||
            ijk[3 * s + 1] >= bx.grid.ny || ijk[3 * s + 2] >= bx.grid.nz)
            return bfail(b, RT_EINVAL, "source outside its box");
        for (int g = 0; g < bx.G; ++g)
            if (!(L[(size_t)s * bx.G + g] >= 0.0) || !std::isfinite(L[(size_t)s * bx.G + g]))
                return bfail(b, RT_EINVAL, "bad source luminosity");
    }
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    bx.src_ijk.assign(ijk, ijk + 3 * n);
    bx.src_L.assign(L, L + (size_t)n * bx.G);
    return upload_sources(b);
}

int rt_batch_courant_dt(const rt_batch *b, double *dt)
{
    if (!b || !dt) return RT_EINVAL;
    *dt = b->opt.cfl * b->dx / (3.0 * b->cr);
    return RT_OK;
}

int rt_batch_step(rt_batch *b, double dt)
{
    if (!b) return RT_EINVAL;
    int rc = bcheck_dt(b, &dt);
    if (rc) return rc;
    return enqueue_batch_step(b, dt);
}

int rt_batch_run(rt_batch *b, double dt, int nsteps)
{
    if (!b) return RT_EINVAL;
    if (nsteps < 0) return bfail(b, RT_EINVAL, "nsteps < 0");
    int rc = bcheck_dt(b, &dt);
    if (rc) return rc;
    if (nsteps == 0) return RT_OK;
    if (!b->graph || b->graph_dt != dt || b->graph_cur0 != b->cur) {
        if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
        cudaGraph_t graph;
        const int cur0 = b->cur;
        B_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        int r1 = enqueue_batch_step(b, dt);
        int r2 = r1 ? r1 : enqueue_batch_step(b, dt);
        cudaError_t ec = cudaStreamEndCapture(b->stream, &graph);
        b->cur = cur0;
        if (r2) return r2;
        if (ec != cudaSuccess) return bcuda(b, ec, "cudaStreamEndCapture");
        cudaError_t ei = cudaGraphInstantiate(&b->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) { b->graph = nullptr; return bcuda(b, ei, "cudaGraphInstantiate"); }
        b->graph_dt = dt;
        b->graph_cur0 = cur0;
    }
    for (int k = 0; k < nsteps / 2; ++k) B_CUDA(b, cudaGraphLaunch(b->graph, b->stream));
    if (nsteps % 2) return enqueue_batch_step(b, dt);
    return RT_OK;
}

int rt_batch_get_budget(rt_batch *b, int box, double *out)
{
    if (!b || !out) return RT_EINVAL;
    if (box < 0 || box >= b->nbox) return bfail(b, RT_EINVAL, "box index out of range");
    int rc = bsync(b);
    B_CUDA(b, cudaMemcpy(out, b->d_budget + 4 * (size_t)b->bg_first[box], 4 * b->box[box].G * sizeof(double),
                         cudaMemcpyDeviceToHost));
    return rc;
}

int rt_batch_sync(rt_batch *b)
{
    if (!b) return RT_EINVAL;
    return bsync(b);
}

const char *rt_batch_last_error(const rt_batch *b)
{
    if (!b) return "null handle";
    return b->err.c_str();
}

int rt_batch_autotune(rt_batch *b, int trials)
{
    if (!b) return RT_EINVAL;
    if (!b->state_set) return bfail(b, RT_EINVAL, "no box state has been set");
    if (trials < 1) trials = 1;
    double dt = b->opt.cfl * b->dx / (3.0 * b->cr);
    std::map<int, std::vector<int>> by_side;
    for (int i = 0; i < b->nbox; ++i)
        by_side[b->box[i].grid.nx * 100000 + b->box[i].grid.ny * 100 + b->box[i].grid.nz].push_back(i);
    const int shapes[2] = {0, 1};
    const int zcs[4] = {4, 8, 16, 32};
    cudaEvent_t e0, e1;
    B_CUDA(b, cudaEventCreate(&e0));
    B_CUDA(b, cudaEventCreate(&e1));
    const void *tab = b->mixed ? (const void *)b->hllf : (const void *)b->hll;
    std::vector<BoxHost> saved = b->box;
    for (auto &kv : by_side) {
        float best = 1e30f;
        int bs = b->box[kv.second[0]].shape, bz = b->box[kv.second[0]].zc;
        for (int sh : shapes) {
            for (int zc : zcs) {
                for (int i = 0; i < b->nbox; ++i) { b->box[i].shape = 2; }   // exclude all
                for (int i : kv.second) { b->box[i].shape = sh; b->box[i].zc = zc; }
                int rc = build_items(b);
                if (rc) { cudaEventDestroy(e0); cudaEventDestroy(e1); return rc; }
                const int nxt = 1 - b->cur;
                float tot = 0.0f;
                for (int t = 0; t <= trials; ++t) {
                    cudaEventRecord(e0, b->stream);
                    launch_transport_batch(b->d_items, b->d_boxes, 0, b->n_items_shape0, 0, b->mixed, b->opt.flux,
                                           b->cr, dt, b->dx, (const void *const *)b->d_Ncls[b->cur],
                                           (const void *const *)b->d_Fcls[b->cur], b->d_Ncls[nxt], b->d_Fcls[nxt],
                                           tab, b->d_pin, b->d_pout, b->stream);
                    launch_transport_batch(b->d_items, b->d_boxes, b->n_items_shape0,
                                           b->n_items - b->n_items_shape0, 1, b->mixed, b->opt.flux, b->cr, dt,
                                           b->dx, (const void *const *)b->d_Ncls[b->cur],
                                           (const void *const *)b->d_Fcls[b->cur], b->d_Ncls[nxt], b->d_Fcls[nxt],
                                           tab, b->d_pin, b->d_pout, b->stream);
                    cudaEventRecord(e1, b->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (t > 0) tot += ms;   // the first launch warms up
                }
                if (tot < best) { best = tot; bs = sh; bz = zc; }
            }
        }
        for (int i = 0; i < b->nbox; ++i) b->box[i] = saved[i];
        for (int i : kv.second) { saved[i].shape = bs; saved[i].zc = bz; b->box[i].shape = bs; b->box[i].zc = bz; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->box = saved;
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    int rc = build_items(b);
    if (rc) return rc;
    B_CUDA(b, cudaStreamSynchronize(b->stream));
    return RT_OK;
}

int rt_batch_box_tiling(const rt_batch *b, int box, int *shape, int *planes)
{
    if (!b || box < 0 || box >= b->nbox || !shape || !planes) return RT_EINVAL;
    *shape = b->box[box].shape;
    *planes = b->box[box].zc;
    return RT_OK;
}

}  // extern "C"

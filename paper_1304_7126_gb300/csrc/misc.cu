// Small kernels of the RT step: point-source injection (paper Sec. 3.1,
// Eq. (injnum)), the reduction of the photons left in the box, and the
// fixed-order finalisation of the photon budget.
#include <cuda_runtime.h>

#include "rt_internal.h"

namespace rtgb {
namespace {

constexpr int RB = 256;       // reduction block
constexpr int RBLK = 296;     // reduction blocks per group (2 per SM)

// N_i += L_i dt / V in each source cell (sources pre-merged per cell); the
// add is done in FP64 and rounded to the state type.
template <typename P>
__global__ void inject_kernel(int nsrc, int G, long long nc, const long long *__restrict__ cells,
                              const double *__restrict__ Lsum, double dt_over_V, P *N)
{
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsrc) return;
    long long c = cells[s];
    for (int g = 0; g < G; ++g) {
        P &n = N[(long long)g * nc + c];
        n = (P)((double)n + Lsum[(long long)s * G + g] * dt_over_V);
    }
}

// x[i] *= f for i < n (the dilution of a change of expansion factor)
template <typename P>
__global__ void scale_kernel(long long n, double f, P *x)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] = (P)((double)x[i] * f);
}

template <typename A, typename B>
__global__ void convert_kernel(long long n, const A *__restrict__ in, B *__restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (B)in[i];
}

__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    __syncthreads();
    return t;   // valid in thread 0
}

// Per-block partial sums of N over the cells of one group; the partition
// of cells into blocks is fixed, so the result is reproducible.
template <typename P>
__global__ void __launch_bounds__(RB) reduce_N_kernel(long long nc, const P *__restrict__ N, double *part)
{
    __shared__ double sh[RB / 32];
    const int g = blockIdx.y;
    const P *Ng = N + (long long)g * nc;
    double acc = 0.0;
    for (long long i = (long long)blockIdx.x * RB + threadIdx.x; i < nc; i += (long long)gridDim.x * RB)
        acc += (double)Ng[i];
    double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(long long)g * gridDim.x + blockIdx.x] = t;
}

__device__ double fixed_sum(const double *a, int n, double *sh)
{
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += a[i];
    return block_sum(acc, sh);
}

struct Emitted {
    double v[kMaxG];
};

// mode 0: after a step; mode 1: at set_state (in_box only, counters zeroed).
__global__ void __launch_bounds__(RB) finalize_kernel(int G, int mode, const double *tr_inbox,
                                                      const double *tr_out, const double *th_inbox,
                                                      int n_tr, int n_red, double V, Emitted em,
                                                      double *budget, unsigned long long *qcounters,
                                                      unsigned *status)
{
    __shared__ double sh[RB / 32];
    for (int g = 0; g < G; ++g) {
        double C = fixed_sum(th_inbox + (long long)g * n_red, n_red, sh);
        double A = 0.0, B = 0.0;
        if (mode == 0) {
            A = fixed_sum(tr_inbox + (long long)g * n_tr, n_tr, sh);
            B = fixed_sum(tr_out + (long long)g * n_tr, n_tr, sh);
        }
        if (threadIdx.x == 0) {
            double *b = budget + 4 * g;
            b[0] = C * V;
            if (mode == 0) {
                b[1] += (A - C) * V;
                b[2] += B;
                b[3] += em.v[g];
            } else {
                b[1] = 0.0;
                b[2] = 0.0;
                b[3] = 0.0;
            }
            if (!isfinite(C) || !isfinite(A) || !isfinite(B)) atomicOr(status, kStatusNonFinite);
        }
    }
    if (threadIdx.x == 0 && qcounters) {
        for (int k = 0; k < kQueueCounters; ++k) qcounters[k] = 0ULL;
    }
}

}  // namespace

int reduce_blocks_per_group() { return RBLK; }

cudaError_t launch_inject(int nsrc, int G, long long nc, const long long *cells, const double *Lsum,
                          double dt_over_V, double *N, cudaStream_t s)
{
    if (nsrc <= 0) return cudaSuccess;
    inject_kernel<double><<<(nsrc + 127) / 128, 128, 0, s>>>(nsrc, G, nc, cells, Lsum, dt_over_V, N);
    return cudaGetLastError();
}

cudaError_t launch_inject_f32(int nsrc, int G, long long nc, const long long *cells, const double *Lsum,
                              double dt_over_V, float *N, cudaStream_t s)
{
    if (nsrc <= 0) return cudaSuccess;
    inject_kernel<float><<<(nsrc + 127) / 128, 128, 0, s>>>(nsrc, G, nc, cells, Lsum, dt_over_V, N);
    return cudaGetLastError();
}

cudaError_t launch_reduce_N(int G, long long nc, const double *N, const Partials &p, cudaStream_t s)
{
    dim3 grid(p.n_red_blocks, G);
    reduce_N_kernel<double><<<grid, RB, 0, s>>>(nc, N, p.th_inbox);
    return cudaGetLastError();
}

cudaError_t launch_reduce_N_f32(int G, long long nc, const float *N, const Partials &p, cudaStream_t s)
{
    dim3 grid(p.n_red_blocks, G);
    reduce_N_kernel<float><<<grid, RB, 0, s>>>(nc, N, p.th_inbox);
    return cudaGetLastError();
}

template <typename P>
static cudaError_t launch_scale_t(long long n, double f, P *x, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    long long b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    scale_kernel<P><<<(unsigned)b, 256, 0, s>>>(n, f, x);
    return cudaGetLastError();
}

cudaError_t launch_scale(long long n, double f, double *x, cudaStream_t s) { return launch_scale_t(n, f, x, s); }
cudaError_t launch_scale_f32(long long n, double f, float *x, cudaStream_t s) { return launch_scale_t(n, f, x, s); }

cudaError_t launch_convert_d2f(long long n, const double *in, float *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    convert_kernel<double, float><<<1216, 256, 0, s>>>(n, in, out);
    return cudaGetLastError();
}

cudaError_t launch_convert_f2d(long long n, const float *in, double *out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    convert_kernel<float, double><<<1216, 256, 0, s>>>(n, in, out);
    return cudaGetLastError();
}

cudaError_t launch_finalize_mode(int G, int mode, const Partials &p, double V, const double *emitted,
                                 double *budget, Queue q, unsigned *status, cudaStream_t s)
{
    Emitted em;
    for (int g = 0; g < kMaxG; ++g) em.v[g] = (g < G && emitted) ? emitted[g] : 0.0;
    finalize_kernel<<<1, RB, 0, s>>>(G, mode, p.tr_inbox, p.tr_outflow, p.th_inbox, p.n_tr_blocks,
                                     p.n_red_blocks, V, em, budget, q.counters, status);
    return cudaGetLastError();
}

}  // namespace rtgb

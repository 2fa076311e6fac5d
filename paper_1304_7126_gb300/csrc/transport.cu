// Photon transport kernel (paper Sec. 3.2): explicit first-order Godunov
// update of U = (N, F) for every photon group,
//     U^{n+1} = U^n + dt/dx * sum_d (Flux_{d, l-1/2} - Flux_{d, l+1/2}),
// unsplit over the six faces (all from U^n), with the M1 closure
// P = c^2 N D(f, n) (Sec. 2, Eqs. (edd2), (eddTens), (Udir)) and the GLF
// (Eq. (glf)) or HLL (Eq. (hll)) intercell flux.
//
// Data layout: N[g][z][y][x], F[g][3][z][y][x], x fastest.  A CTA works on
// 32 x 8 (x, y) tiles of one group, marching along z; a single box runs a
// persistent grid whose CTAs each take an equal contiguous range of the
// (group, tile, plane) units.  Each thread keeps its own column's cells
// z-1, z, z+1 in registers, so the closure is evaluated once per cell and
// every z face flux once; the in-plane neighbours (and the one-cell halo
// ring of the tile, recomputed by the ring threads) go through shared
// memory, where every x and y face flux is also evaluated once.  Reads and
// writes of the planes are coalesced 256-byte rows.  Per-CTA photon sums
// (in the box after transport, net outflow through boundary faces) go to a
// partials array reduced later in a fixed order, so the budget is
// reproducible for a given grid.
//
// The kernel is templated on the state type S: double (the FP64 path) or
// float (the mixed path, RT_MIXED: state stored and transported in FP32,
// half the HBM traffic; the six face-flux differences are added to U with
// error-free TwoSum steps and the accumulated rounding error folded back in
// once, so an update loses one rounding instead of several).
#include <cuda_runtime.h>

#include "rt_internal.h"

namespace rtgb {
namespace {

template <typename S>
struct CellQ {
    S N, Fx, Fy, Fz;            // U
    S Pxx, Pxy, Pxz, Pyy, Pyz, Pzz;   // c^2 N D
    S lmin[3], lmax[3];         // HLL wave speeds (already times c)
};

template <typename S> struct Vec2;
template <> struct Vec2<double> { using T = double2; };
template <> struct Vec2<float> { using T = float2; };

// Every product, sum and fused multiply-add below is written out with a
// rounded intrinsic, so the compiler fuses nothing on its own: the
// single-box and batched kernels, which inline the same code in different
// surroundings, then give the same bits.
__device__ __forceinline__ double tmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float tmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double tadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float tadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double tsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float tsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double tfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float tfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// 1/d for d > 0: in FP64 an FP32 reciprocal of d (the conversions through
// integer operations, so nothing but the Newton steps uses the FP64 pipe)
// refined by two Newton steps (within an ulp; the FP64 transport is bound
// by its FP64 instructions, and the IEEE quotient takes about twice as
// many); d outside the float range takes the IEEE quotient.  In FP32 the
// hardware's approximate reciprocal.
__device__ __forceinline__ float f32_of(double x)   // nearest float, x a normal float magnitude
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long a = (b & 0x7fffffffffffffffULL) + 0x10000000ULL;
    return __uint_as_float(((unsigned)(b >> 63) << 31) | ((unsigned)((a >> 52) - 896) << 23) |
                           (unsigned)((a >> 29) & 0x7fffff));
}
__device__ __forceinline__ double f64_of(float f)   // exact, f a normal float
{
    const unsigned u = __float_as_uint(f);
    return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                            ((unsigned long long)(((u >> 23) & 0xff) + 896) << 52) |
                                            ((unsigned long long)(u & 0x7fffff) << 29)));
}
__device__ __forceinline__ double trcp(double d)
{
    const unsigned long long e = ((unsigned long long)__double_as_longlong(d) >> 52) & 0x7ff;
    if (e < 1023 - 120 || e > 1023 + 120) return 1.0 / d;   // |d| outside [2^-120, 2^121)
    double r = f64_of(__fdividef(1.0f, f32_of(d)));
    r = __fma_rn(r, __fma_rn(-d, r, 1.0), r);
    return __fma_rn(r, __fma_rn(-d, r, 1.0), r);
}
__device__ __forceinline__ float trcp(float d) { return __fdividef(1.0f, d); }

template <typename S>
__device__ __forceinline__ void hll_lookup(const S *__restrict__ tab, S f, S mu, S &lo, S &hi)
{
    S fx = tmul(f, (S)(kHllNF - 1));
    int k = (int)floor(fx);
    k = k < 0 ? 0 : (k > kHllNF - 2 ? kHllNF - 2 : k);
    S wf = tsub(fx, (S)k);
    S mx = tmul(tadd(mu, (S)1), (S)(0.5 * (kHllNMU - 1)));
    int j = (int)floor(mx);
    j = j < 0 ? 0 : (j > kHllNMU - 2 ? kHllNMU - 2 : j);
    S wm = tsub(mx, (S)j);
    using V = typename Vec2<S>::T;
    const V *t = reinterpret_cast<const V *>(tab);
    V a = __ldg(&t[k * kHllNMU + j]);
    V b = __ldg(&t[k * kHllNMU + j + 1]);
    V c = __ldg(&t[(k + 1) * kHllNMU + j]);
    V d = __ldg(&t[(k + 1) * kHllNMU + j + 1]);
    S lo0 = tfma(wm, tsub(b.x, a.x), a.x), lo1 = tfma(wm, tsub(d.x, c.x), c.x);
    S hi0 = tfma(wm, tsub(b.y, a.y), a.y), hi1 = tfma(wm, tsub(d.y, c.y), c.y);
    lo = tfma(wf, tsub(lo1, lo0), lo0);
    hi = tfma(wf, tsub(hi1, hi0), hi0);
}

// Photon densities below this are no photons: the closure takes f = 0.
constexpr double kClosureFloorN = 1e-30;

// M1 closure of one cell.  f := 0 for F = 0 or N below kClosureFloorN; f
// clamped to 1.  In FP32, F is scaled by a power of two (exact) for the
// direction and |F| so that its square neither underflows for N down to the
// floor nor overflows.
template <typename S, int FLUX>
__device__ __forceinline__ void closure(S N, S Fx, S Fy, S Fz, S c, const S *__restrict__ tab, CellQ<S> &q)
{
    q.N = N; q.Fx = Fx; q.Fy = Fy; q.Fz = Fz;
    S sc = (S)1;
    if (sizeof(S) != sizeof(double)) {
        S m = fmax(fabs(Fx), fmax(fabs(Fy), fabs(Fz)));
        sc = (m < (S)1e-15) ? (S)0x1p64 : ((m > (S)1e15) ? (S)0x1p-64 : (S)1);
    }
    const S gx = tmul(Fx, sc), gy = tmul(Fy, sc), gz = tmul(Fz, sc);
    S F2 = tfma(gz, gz, tfma(gy, gy, tmul(gx, gx)));
    S f = 0, nx = 0, ny = 0, nz = 0;
    if (N > (S)kClosureFloorN && F2 > (S)0) {
        S inv = rsqrt(F2);
        f = fmin(tmul(tmul(F2, inv), trcp(tmul(tmul(c, N), sc))), (S)1);
        nx = tmul(gx, inv); ny = tmul(gy, inv); nz = tmul(gz, inv);
    }
    S f2 = tmul(f, f);
    S chi = tmul(tfma((S)4, f2, (S)3), trcp(tfma((S)2, sqrt(tfma((S)-3, f2, (S)4)), (S)5)));
    S cN = tmul(tmul(c, c), N);
    S ch = tmul(cN, (S)0.5);
    S ca = tmul(ch, tsub((S)1, chi));
    S cb = tmul(ch, tfma((S)3, chi, (S)-1));
    S bx = tmul(cb, nx), by = tmul(cb, ny);
    q.Pxx = tfma(bx, nx, ca);
    q.Pyy = tfma(by, ny, ca);
    q.Pzz = tfma(tmul(cb, nz), nz, ca);
    q.Pxy = tmul(bx, ny);
    q.Pxz = tmul(bx, nz);
    q.Pyz = tmul(by, nz);
    if (FLUX == RT_HLL) {
        S lo, hi;
        hll_lookup<S>(tab, f, nx, lo, hi); q.lmin[0] = tmul(lo, c); q.lmax[0] = tmul(hi, c);
        hll_lookup<S>(tab, f, ny, lo, hi); q.lmin[1] = tmul(lo, c); q.lmax[1] = tmul(hi, c);
        hll_lookup<S>(tab, f, nz, lo, hi); q.lmin[2] = tmul(lo, c); q.lmax[2] = tmul(hi, c);
    }
}

// Intercell flux along direction D from left cell L to right cell R.
template <typename S, int FLUX, int D>
__device__ __forceinline__ void face_flux(const CellQ<S> &L, const CellQ<S> &R, S c, S out[4])
{
    S fl[4], fr[4], ul[4], ur[4];
    ul[0] = L.N; ul[1] = L.Fx; ul[2] = L.Fy; ul[3] = L.Fz;
    ur[0] = R.N; ur[1] = R.Fx; ur[2] = R.Fy; ur[3] = R.Fz;
    if (D == 0) {
        fl[0] = L.Fx; fl[1] = L.Pxx; fl[2] = L.Pxy; fl[3] = L.Pxz;
        fr[0] = R.Fx; fr[1] = R.Pxx; fr[2] = R.Pxy; fr[3] = R.Pxz;
    } else if (D == 1) {
        fl[0] = L.Fy; fl[1] = L.Pxy; fl[2] = L.Pyy; fl[3] = L.Pyz;
        fr[0] = R.Fy; fr[1] = R.Pxy; fr[2] = R.Pyy; fr[3] = R.Pyz;
    } else {
        fl[0] = L.Fz; fl[1] = L.Pxz; fl[2] = L.Pyz; fl[3] = L.Pzz;
        fr[0] = R.Fz; fr[1] = R.Pxz; fr[2] = R.Pyz; fr[3] = R.Pzz;
    }
    if (FLUX == RT_HLL) {
        S lp = fmax((S)0, fmax(L.lmax[D], R.lmax[D]));
        S lm = fmin((S)0, fmin(L.lmin[D], R.lmin[D]));
        S den = tsub(lp, lm);
        if (den > (S)0) {
            S inv = trcp(den);
            S pm = tmul(lp, lm);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                out[k] = tmul(tfma(pm, tsub(ur[k], ul[k]), tfma(-lm, fr[k], tmul(lp, fl[k]))), inv);
        } else {
            // both speeds vanish only for f = 1 beams parallel to the face
#pragma unroll
            for (int k = 0; k < 4; ++k) out[k] = tmul((S)0.5, tadd(fl[k], fr[k]));
        }
    } else {
        const S hc = tmul((S)0.5, c);
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = tfma(-hc, tsub(ur[k], ul[k]), tmul((S)0.5, tadd(fl[k], fr[k])));
    }
}

// Error-free sum a + b = s + e (Knuth's TwoSum), FP32; the _rn intrinsics
// keep the compiler from contracting the steps into FMAs.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// A thread's share of the budget sums (photons left in the box, boundary
// outflow): a double in the FP64 path; in the FP32 path a float pair summed
// with TwoSum (no FP64 instruction per cell; exact to ~2^-48), widened once
// per tile.
template <typename S> struct BudgetAcc;
template <> struct BudgetAcc<double> {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ double get() const { return v; }
};
template <> struct BudgetAcc<float> {
    float s = 0.0f, e = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        float t, r;
        two_sum(s, x, t, r);
        s = t;
        e = __fadd_rn(e, r);
    }
    __device__ __forceinline__ double get() const { return (double)s + (double)e; }
};

// Load U at (x, y, z) where at most one coordinate may sit one cell outside
// the box: that position is the boundary ghost (outflow: copy; reflect:
// copy with the normal flux negated; periodic: wrap; inflow: the face's
// given state).
// inf: this group's inflow ghost states [6 faces][N, Fx, Fy, Fz], or NULL
template <typename S>
__device__ __forceinline__ void load_U(const GridDev &g, const S *__restrict__ N, const S *__restrict__ F,
                                       const S *__restrict__ inf, int x, int y, int z, S &n, S &fx, S &fy, S &fz)
{
    // a face held at a given state (RT_BC_INFLOW)
    int face = -1;
    if (x < 0) face = 0; else if (x >= g.nx) face = 1;
    else if (y < 0) face = 2; else if (y >= g.ny) face = 3;
    else if (z < 0) face = 4; else if (z >= g.nz) face = 5;
    if (face >= 0 && g.bc[face] == RT_BC_INFLOW) {
        if (inf) {
            n = inf[4 * face]; fx = inf[4 * face + 1]; fy = inf[4 * face + 2]; fz = inf[4 * face + 3];
        } else {
            n = fx = fy = fz = (S)0;
        }
        return;
    }
    int flip = -1;
    if (x < 0) {
        if (g.bc[0] == RT_BC_PERIODIC) x = g.nx - 1; else { x = 0; if (g.bc[0] == RT_BC_REFLECT) flip = 0; }
    } else if (x >= g.nx) {
        if (g.bc[1] == RT_BC_PERIODIC) x = 0; else { x = g.nx - 1; if (g.bc[1] == RT_BC_REFLECT) flip = 0; }
    }
    if (y < 0) {
        if (g.bc[2] == RT_BC_PERIODIC) y = g.ny - 1; else { y = 0; if (g.bc[2] == RT_BC_REFLECT) flip = 1; }
    } else if (y >= g.ny) {
        if (g.bc[3] == RT_BC_PERIODIC) y = 0; else { y = g.ny - 1; if (g.bc[3] == RT_BC_REFLECT) flip = 1; }
    }
    if (z < 0) {
        if (g.bc[4] == RT_BC_PERIODIC) z = g.nz - 1; else { z = 0; if (g.bc[4] == RT_BC_REFLECT) flip = 2; }
    } else if (z >= g.nz) {
        if (g.bc[5] == RT_BC_PERIODIC) z = 0; else { z = g.nz - 1; if (g.bc[5] == RT_BC_REFLECT) flip = 2; }
    }
    long long i = ((long long)z * g.ny + y) * g.nx + x;
    n = __ldg(&N[i]);
    fx = __ldg(&F[i]);
    fy = __ldg(&F[g.stride + i]);
    fz = __ldg(&F[2 * g.stride + i]);
    if (flip == 0) fx = -fx;
    if (flip == 1) fy = -fy;
    if (flip == 2) fz = -fz;
}

// Shared-memory plane of closure quantities needed by the x and y faces.
template <typename S, int TBX, int TBY>
struct PlaneSmem {
    static constexpr int SW = TBX + 2, SH = TBY + 2;
    S N[SH][SW], Fx[SH][SW], Fy[SH][SW], Fz[SH][SW];
    S Pxx[SH][SW], Pxy[SH][SW], Pxz[SH][SW], Pyy[SH][SW], Pyz[SH][SW];
    S lminx[SH][SW], lmaxx[SH][SW], lminy[SH][SW], lmaxy[SH][SW];
    S fxs[4][TBY][TBX + 1];     // x faces 0..TBX of each row
    S fys[4][TBY + 1][TBX];     // y faces 0..TBY of each column
    double red[2][TBX * TBY / 32];
};

template <typename S, int FLUX, class SM>
__device__ __forceinline__ void put_plane(SM &s, int r, int c, const CellQ<S> &q)
{
    s.N[r][c] = q.N; s.Fx[r][c] = q.Fx; s.Fy[r][c] = q.Fy; s.Fz[r][c] = q.Fz;
    s.Pxx[r][c] = q.Pxx; s.Pxy[r][c] = q.Pxy; s.Pxz[r][c] = q.Pxz; s.Pyy[r][c] = q.Pyy; s.Pyz[r][c] = q.Pyz;
    if (FLUX == RT_HLL) {
        s.lminx[r][c] = q.lmin[0]; s.lmaxx[r][c] = q.lmax[0];
        s.lminy[r][c] = q.lmin[1]; s.lmaxy[r][c] = q.lmax[1];
    }
}

template <typename S, int FLUX, class SM>
__device__ __forceinline__ void get_plane(const SM &s, int r, int c, CellQ<S> &q)
{
    q.N = s.N[r][c]; q.Fx = s.Fx[r][c]; q.Fy = s.Fy[r][c]; q.Fz = s.Fz[r][c];
    q.Pxx = s.Pxx[r][c]; q.Pxy = s.Pxy[r][c]; q.Pxz = s.Pxz[r][c]; q.Pyy = s.Pyy[r][c]; q.Pyz = s.Pyz[r][c];
    q.Pzz = 0;
    if (FLUX == RT_HLL) {
        q.lmin[0] = s.lminx[r][c]; q.lmax[0] = s.lmaxx[r][c];
        q.lmin[1] = s.lminy[r][c]; q.lmax[1] = s.lmaxy[r][c];
        q.lmin[2] = 0; q.lmax[2] = 0;
    }
}

// One tile of one group: the (x0.., y0..) TBX x TBY column block of planes
// z0 <= z < z1 of a box g, state at N0/F0 (group base pointers, component
// stride g.stride), result to N1/F1.  Returns this thread's share of the
// photons left in the box (sum N) and of the net boundary outflow (flux).
template <typename S, int FLUX, int TBX, int TBY>
__device__ __forceinline__ void transport_tile(PlaneSmem<S, TBX, TBY> &s, const GridDev &g, S c, S dtdx,
                                               const S *__restrict__ N0, const S *__restrict__ F0,
                                               S *__restrict__ N1, S *__restrict__ F1, const S *__restrict__ tab,
                                               const S *__restrict__ inf, int x0, int y0, int z0, int z1,
                                               double &inbox, double &outflow)
{
    // (tx, ty) from the linear thread index: 2-D blocks of TBX x TBY or 1-D
    // blocks of TBX * TBY threads alike
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int tx = tid % TBX, ty = tid / TBX;
    const int x = x0 + tx, y = y0 + ty;
    const bool active = (x < g.nx) && (y < g.ny);
    // ghost-only position of this thread's smem slot (ragged tile edge)
    const bool ghost_slot = !active && ((x == g.nx && y < g.ny) || (x < g.nx && y == g.ny));
    const bool bc_x_lo = g.bc[0] != RT_BC_PERIODIC, bc_x_hi = g.bc[1] != RT_BC_PERIODIC;
    const bool bc_y_lo = g.bc[2] != RT_BC_PERIODIC, bc_y_hi = g.bc[3] != RT_BC_PERIODIC;
    const bool bc_z_lo = g.bc[4] != RT_BC_PERIODIC, bc_z_hi = g.bc[5] != RT_BC_PERIODIC;

    // halo ring slot of this thread (80 slots: left/right columns, bottom/top rows)
    int hr = -1, hc = -1, hx = 0, hy = 0;
    bool hvalid = false;
    if (tid < 2 * TBY) {
        int r = tid % TBY, side = tid / TBY;
        hr = r + 1; hc = side ? TBX + 1 : 0;
        hx = side ? x0 + TBX : x0 - 1; hy = y0 + r;
        hvalid = hy < g.ny && hx <= g.nx;
    } else if (tid < 2 * TBY + 2 * TBX) {
        int t = tid - 2 * TBY;
        int cc = t % TBX, side = t / TBX;
        hr = side ? TBY + 1 : 0; hc = cc + 1;
        hx = x0 + cc; hy = side ? y0 + TBY : y0 - 1;
        hvalid = hx < g.nx && hy <= g.ny;
    }

    CellQ<S> cur, nxt;
    S flo[4] = {0, 0, 0, 0}, fhi[4] = {0, 0, 0, 0};
    BudgetAcc<S> in_acc, out_acc;
    if (active) {
        S n, fx, fy, fz;
        load_U<S>(g, N0, F0, inf, x, y, z0 - 1, n, fx, fy, fz);
        CellQ<S> prev;
        closure<S, FLUX>(n, fx, fy, fz, c, tab, prev);
        load_U<S>(g, N0, F0, inf, x, y, z0, n, fx, fy, fz);
        closure<S, FLUX>(n, fx, fy, fz, c, tab, cur);
        face_flux<S, FLUX, 2>(prev, cur, c, flo);
    }

    for (int z = z0; z < z1; ++z) {
        if (active) {
            S n, fx, fy, fz;
            load_U<S>(g, N0, F0, inf, x, y, z + 1, n, fx, fy, fz);
            closure<S, FLUX>(n, fx, fy, fz, c, tab, nxt);
            face_flux<S, FLUX, 2>(cur, nxt, c, fhi);
            put_plane<S, FLUX>(s, ty + 1, tx + 1, cur);
        } else if (ghost_slot) {
            S n, fx, fy, fz;
            CellQ<S> q;
            load_U<S>(g, N0, F0, inf, x, y, z, n, fx, fy, fz);
            closure<S, FLUX>(n, fx, fy, fz, c, tab, q);
            put_plane<S, FLUX>(s, ty + 1, tx + 1, q);
        }
        if (hvalid) {
            S n, fx, fy, fz;
            CellQ<S> q;
            load_U<S>(g, N0, F0, inf, hx, hy, z, n, fx, fy, fz);
            closure<S, FLUX>(n, fx, fy, fz, c, tab, q);
            put_plane<S, FLUX>(s, hr, hc, q);
        }
        __syncthreads();

        // x face ff of row r lies between smem columns ff and ff + 1, at
        // global x position x0 + ff - 1/2; y face ff of column cx between
        // smem rows ff and ff + 1.  Thread (tx, ty) takes x face tx of row ty
        // and y face ty of column tx; the tile's far faces (x face TBX of
        // each row, y face TBY of each column) go to warps of their own in a
        // second pass of each (no warp runs a face pass for one lane).
        constexpr int kFarX = ((TBX + 31) / 32) * 32;   // first thread of the far x faces
        static_assert(kFarX + TBY <= TBX * TBY, "far faces need TBX + TBY threads in separate warps");
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
            int r = ty, ff = tx;   // x face ff of row r
            bool on = y < g.ny;
            if (q == 1) {
                r = tid - kFarX;
                ff = TBX;
                on = tid >= kFarX && tid < kFarX + TBY && y0 + r < g.ny;
            }
            const int gxf = x0 + ff;
            if (on && gxf <= g.nx) {
                CellQ<S> L, R;
                get_plane<S, FLUX>(s, r + 1, ff, L);
                get_plane<S, FLUX>(s, r + 1, ff + 1, R);
                S fl[4];
                face_flux<S, FLUX, 0>(L, R, c, fl);
#pragma unroll
                for (int k = 0; k < 4; ++k) s.fxs[k][r][ff] = fl[k];
                if (gxf == 0 && bc_x_lo) out_acc.add(-fl[0]);
                if (gxf == g.nx && bc_x_hi) out_acc.add(fl[0]);
            }
        }
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
            int cx = tx, ff = ty;   // y face ff of column cx
            bool on = x < g.nx;
            if (q == 1) {
                cx = tid;
                ff = TBY;
                on = tid < TBX && x0 + cx < g.nx;
            }
            const int gyf = y0 + ff;
            if (on && gyf <= g.ny) {
                CellQ<S> L, R;
                get_plane<S, FLUX>(s, ff, cx + 1, L);
                get_plane<S, FLUX>(s, ff + 1, cx + 1, R);
                S fl[4];
                face_flux<S, FLUX, 1>(L, R, c, fl);
#pragma unroll
                for (int k = 0; k < 4; ++k) s.fys[k][ff][cx] = fl[k];
                if (gyf == 0 && bc_y_lo) out_acc.add(-fl[0]);
                if (gyf == g.ny && bc_y_hi) out_acc.add(fl[0]);
            }
        }
        __syncthreads();

        if (active) {
            S u[4] = {cur.N, cur.Fx, cur.Fy, cur.Fz};
            S nw[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (sizeof(S) == sizeof(double)) {
                    S acc = tadd(tadd(tsub(s.fxs[k][ty][tx], s.fxs[k][ty][tx + 1]),
                                      tsub(s.fys[k][ty][tx], s.fys[k][ty + 1][tx])),
                                 tsub(flo[k], fhi[k]));
                    nw[k] = tfma(dtdx, acc, u[k]);
                } else {
                    // compensated: U + sum of six dt/dx-scaled face fluxes
                    float d = (float)dtdx;
                    float t[6] = {__fmul_rn(d, (float)s.fxs[k][ty][tx]), -__fmul_rn(d, (float)s.fxs[k][ty][tx + 1]),
                                  __fmul_rn(d, (float)s.fys[k][ty][tx]), -__fmul_rn(d, (float)s.fys[k][ty + 1][tx]),
                                  __fmul_rn(d, (float)flo[k]), -__fmul_rn(d, (float)fhi[k])};
                    float sum = (float)u[k], err = 0.0f;
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        float e;
                        two_sum(sum, t[q], sum, e);
                        err = __fadd_rn(err, e);
                    }
                    nw[k] = (S)__fadd_rn(sum, err);
                }
            }
            // realisability |F| <= c N (acts only at rounding level for CFL <= 1)
            if (nw[0] < (S)0) { nw[0] = 0; nw[1] = nw[2] = nw[3] = 0; }
            // squares of tiny values lose digits: compare tiny states scaled
            // by a power of two (exact), the factor is scale-free
            S cn = tmul(c, nw[0]);
            S m = fmax(fmax(fabs(nw[1]), fabs(nw[2])), fmax(fabs(nw[3]), cn));
            const S tiny = sizeof(S) == sizeof(double) ? (S)1e-140 : (S)1e-15;
            const S big = sizeof(S) == sizeof(double) ? (S)0x1p600 : (S)0x1p60;
            S sc0 = (m < tiny) ? big : (S)1;
            S f1 = tmul(nw[1], sc0), f2 = tmul(nw[2], sc0), f3 = tmul(nw[3], sc0), cs = tmul(cn, sc0);
            S F2 = tfma(f3, f3, tfma(f2, f2, tmul(f1, f1)));
            if (F2 > tmul(cs, cs)) {
                S sc = (F2 > (S)0) ? tmul(cs, rsqrt(F2)) : (S)0;
                nw[1] = tmul(nw[1], sc); nw[2] = tmul(nw[2], sc); nw[3] = tmul(nw[3], sc);
            }
            long long i = ((long long)z * g.ny + y) * g.nx + x;
            N1[i] = nw[0];
            F1[i] = nw[1];
            F1[g.stride + i] = nw[2];
            F1[2 * g.stride + i] = nw[3];
            in_acc.add(nw[0]);
            if (z == 0 && bc_z_lo) out_acc.add(-flo[0]);
            if (z == g.nz - 1 && bc_z_hi) out_acc.add(fhi[0]);
            cur = nxt;
#pragma unroll
            for (int k = 0; k < 4; ++k) flo[k] = fhi[k];
        }
        __syncthreads();
    }
    inbox = in_acc.get();
    outflow = out_acc.get();
}

// fixed-order block reduction of the two budget sums (thread 0 gets them)
template <int NT>
__device__ __forceinline__ void block_reduce2(double *red, double &a, double &b)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int warp = tid >> 5, lane = tid & 31;
    if (lane == 0) { red[warp] = a; red[NT / 32 + warp] = b; }
    __syncthreads();
    if (tid == 0) {
        double x = 0.0, y = 0.0;
        for (int w = 0; w < NT / 32; ++w) { x += red[w]; y += red[NT / 32 + w]; }
        a = x;
        b = y;
    }
}

// one column segment of the persistent kernel, out of line: inlined into the
// segment loop it spilled registers inside the plane loop
template <typename S, int FLUX, int TBX, int TBY>
__device__ __noinline__ void transport_segment(PlaneSmem<S, TBX, TBY> &s, const GridDev &g, S c, S dtdx,
                                               const S *__restrict__ N0, const S *__restrict__ F0,
                                               S *__restrict__ N1, S *__restrict__ F1, const S *__restrict__ tab,
                                               const S *__restrict__ inf, int x0, int y0, int z0, int z1,
                                               double &inbox, double &outflow)
{
    transport_tile<S, FLUX, TBX, TBY>(s, g, c, dtdx, N0, F0, N1, F1, tab, inf, x0, y0, z0, z1, inbox, outflow);
}

// Single box: a persistent grid (transport_grid: 2 CTAs per SM in FP64, 4 in FP32).  The
// (group, tile, plane) units, planes fastest, are cut into gridDim.x equal
// contiguous ranges, one per CTA, so every CTA gets the same number of
// planes (a launch of one CTA per tile chunk left a last, nearly empty wave);
// a CTA walks its range one tile column segment at a time.  Budget partials:
// [group][CTA], each the CTA's segments of that group summed in order.
template <typename S, int FLUX>
__device__ __forceinline__ void transport_kernel_body(GridDev g, int G, S c, S dtdx, double area_dt,
                                                      const S *__restrict__ N0all, const S *__restrict__ F0all,
                                                      S *__restrict__ N1all, S *__restrict__ F1all,
                                                      const S *__restrict__ tab, const S *__restrict__ inflow,
                                                      double *__restrict__ part_inbox,
                                                      double *__restrict__ part_out, int tiles_x, int tiles_y)
{
    constexpr int TBX = 32, TBY = 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PlaneSmem<S, TBX, TBY> &s = *reinterpret_cast<PlaneSmem<S, TBX, TBY> *>(smem_raw);
    const long long tiles = (long long)tiles_x * tiles_y;
    const long long units = tiles * G * g.nz;
    const long long u1 = units * (blockIdx.x + 1) / gridDim.x;
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    // the range visits the groups in increasing order: the sums of the
    // current one are kept, written when the group changes (every group's
    // slot is zeroed first)
    if (lead)
        for (int k = 0; k < G; ++k) part_inbox[(long long)k * gridDim.x + blockIdx.x] = part_out[(long long)k * gridDim.x + blockIdx.x] = 0.0;
    int cur = -1;
    double acc_in = 0.0, acc_out = 0.0;
    for (long long u = units * blockIdx.x / gridDim.x; u < u1;) {
        const long long col = u / g.nz;
        const int z0 = (int)(u - col * g.nz);
        const int z1 = (int)min((long long)g.nz, z0 + (u1 - u));
        const int grp = (int)(col / tiles);
        const int tile = (int)(col - grp * tiles);
        double inbox, outflow;
        transport_segment<S, FLUX, TBX, TBY>(s, g, c, dtdx, N0all + (long long)grp * g.stride,
                                             F0all + 3LL * grp * g.stride, N1all + (long long)grp * g.stride,
                                             F1all + 3LL * grp * g.stride, tab, inflow ? inflow + 24 * grp : nullptr,
                                             (tile % tiles_x) * TBX, (tile / tiles_x) * TBY, z0, z1, inbox, outflow);
        block_reduce2<TBX * TBY>(&s.red[0][0], inbox, outflow);
        if (lead) {
            if (grp != cur && cur >= 0) {
                part_inbox[(long long)cur * gridDim.x + blockIdx.x] = acc_in;
                part_out[(long long)cur * gridDim.x + blockIdx.x] = acc_out * area_dt;
                acc_in = acc_out = 0.0;
            }
            cur = grp;
            acc_in += inbox;
            acc_out += outflow;
        }
        __syncthreads();
        u += z1 - z0;
    }
    if (lead && cur >= 0) {
        part_inbox[(long long)cur * gridDim.x + blockIdx.x] = acc_in;
        part_out[(long long)cur * gridDim.x + blockIdx.x] = acc_out * area_dt;
    }
}

// FP64: capped at 128 registers so that two CTAs share an SM.  FP32: capped at 64
// registers so that four CTAs share an SM and hide the shared-memory and
// table-lookup latencies (the FP32 kernel is latency-bound; 2, 3 and 4 CTAs
// per SM gave 0.39, 0.35 and 0.33 ms at 128^3 x 3 groups).
template <typename S, int FLUX>
__global__ void __launch_bounds__(256, 2)
transport_kernel(GridDev g, int G, S c, S dtdx, double area_dt, const S *__restrict__ N0all,
                 const S *__restrict__ F0all, S *__restrict__ N1all, S *__restrict__ F1all,
                 const S *__restrict__ tab, const S *__restrict__ inflow, double *__restrict__ part_inbox,
                 double *__restrict__ part_out, int tiles_x, int tiles_y)
{
    transport_kernel_body<S, FLUX>(g, G, c, dtdx, area_dt, N0all, F0all, N1all, F1all, tab, inflow, part_inbox,
                                   part_out, tiles_x, tiles_y);
}

template <int FLUX>
__global__ void __launch_bounds__(256, 4)
transport_kernel_f32(GridDev g, int G, float c, float dtdx, double area_dt, const float *__restrict__ N0all,
                     const float *__restrict__ F0all, float *__restrict__ N1all, float *__restrict__ F1all,
                     const float *__restrict__ tab, const float *__restrict__ inflow,
                     double *__restrict__ part_inbox, double *__restrict__ part_out, int tiles_x, int tiles_y)
{
    transport_kernel_body<float, FLUX>(g, G, c, dtdx, area_dt, N0all, F0all, N1all, F1all, tab, inflow,
                                       part_inbox, part_out, tiles_x, tiles_y);
}

// Batched boxes: CTA i works on item i (box, group, tile, z range) of a
// work list; every box is described by its GridDev (component stride = the
// stride of its group class) and the offset of its first cell in the class.
template <typename S, int FLUX, int TBX, int TBY>
__global__ void __launch_bounds__(TBX * TBY)
transport_batch_kernel(const BatchItem *__restrict__ items, const BatchBox *__restrict__ boxes, S c, S dtdx,
                       double area_dt, const S *const *__restrict__ N0cls, const S *const *__restrict__ F0cls,
                       S *const *__restrict__ N1cls, S *const *__restrict__ F1cls, const S *__restrict__ tab,
                       double *__restrict__ part_inbox, double *__restrict__ part_out, int item0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PlaneSmem<S, TBX, TBY> &s = *reinterpret_cast<PlaneSmem<S, TBX, TBY> *>(smem_raw);
    const int it = item0 + blockIdx.x;
    const BatchItem w = items[it];
    const BatchBox b = boxes[w.box];
    const long long base = (long long)w.grp * b.g.stride + b.cell_off;
    const long long fbase = 3LL * w.grp * b.g.stride + b.cell_off;
    double inbox, outflow;
    transport_tile<S, FLUX, TBX, TBY>(s, b.g, c, dtdx, N0cls[b.cls] + base, F0cls[b.cls] + fbase,
                                      N1cls[b.cls] + base, F1cls[b.cls] + fbase, tab, nullptr, w.x0, w.y0, w.z0,
                                      w.z1, inbox, outflow);
    block_reduce2<TBX * TBY>(&s.red[0][0], inbox, outflow);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        part_inbox[it] = inbox;
        part_out[it] = outflow * area_dt;
    }
}

// The same over both tile shapes in one launch: CTAs [0, n_shape0) take the
// 32 x 8 items, the rest the 16 x 16 ones (1-D blocks of 256 threads, the
// larger of the two shared-memory layouts).
template <typename S, int FLUX>
__global__ void __launch_bounds__(256)
transport_batch_all_kernel(const BatchItem *__restrict__ items, const BatchBox *__restrict__ boxes, S c, S dtdx,
                           double area_dt, const S *const *__restrict__ N0cls, const S *const *__restrict__ F0cls,
                           S *const *__restrict__ N1cls, S *const *__restrict__ F1cls, const S *__restrict__ tab,
                           double *__restrict__ part_inbox, double *__restrict__ part_out, int n_shape0)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int it = blockIdx.x;
    const BatchItem w = items[it];
    const BatchBox b = boxes[w.box];
    const long long base = (long long)w.grp * b.g.stride + b.cell_off;
    const long long fbase = 3LL * w.grp * b.g.stride + b.cell_off;
    double inbox, outflow;
    if (it < n_shape0) {
        PlaneSmem<S, 32, 8> &s = *reinterpret_cast<PlaneSmem<S, 32, 8> *>(smem_raw);
        transport_tile<S, FLUX, 32, 8>(s, b.g, c, dtdx, N0cls[b.cls] + base, F0cls[b.cls] + fbase,
                                       N1cls[b.cls] + base, F1cls[b.cls] + fbase, tab, nullptr, w.x0, w.y0, w.z0,
                                       w.z1, inbox, outflow);
        block_reduce2<256>(&s.red[0][0], inbox, outflow);
    } else {
        PlaneSmem<S, 16, 16> &s = *reinterpret_cast<PlaneSmem<S, 16, 16> *>(smem_raw);
        transport_tile<S, FLUX, 16, 16>(s, b.g, c, dtdx, N0cls[b.cls] + base, F0cls[b.cls] + fbase,
                                        N1cls[b.cls] + base, F1cls[b.cls] + fbase, tab, nullptr, w.x0, w.y0, w.z0,
                                        w.z1, inbox, outflow);
        block_reduce2<256>(&s.red[0][0], inbox, outflow);
    }
    if (threadIdx.x == 0) {
        part_inbox[it] = inbox;
        part_out[it] = outflow * area_dt;
    }
}

template <typename S>
constexpr int batch_all_smem()
{
    return (int)(sizeof(PlaneSmem<S, 32, 8>) > sizeof(PlaneSmem<S, 16, 16>) ? sizeof(PlaneSmem<S, 32, 8>)
                                                                             : sizeof(PlaneSmem<S, 16, 16>));
}

}  // namespace

int transport_grid(int n_sm, bool fp32)
{
    return (fp32 ? 4 : 2) * (n_sm > 0 ? n_sm : 1);
}

template <typename S, int TBX, int TBY>
static void set_smem_attr_batch()
{
    int sz = (int)sizeof(PlaneSmem<S, TBX, TBY>);
    cudaFuncSetAttribute(transport_batch_kernel<S, RT_HLL, TBX, TBY>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz);
    cudaFuncSetAttribute(transport_batch_kernel<S, RT_GLF, TBX, TBY>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz);
}

void transport_init()
{
    int s8 = (int)sizeof(PlaneSmem<double, 32, 8>), s4 = (int)sizeof(PlaneSmem<float, 32, 8>);
    cudaFuncSetAttribute(transport_kernel<double, RT_HLL>, cudaFuncAttributeMaxDynamicSharedMemorySize, s8);
    cudaFuncSetAttribute(transport_kernel<double, RT_GLF>, cudaFuncAttributeMaxDynamicSharedMemorySize, s8);
    cudaFuncSetAttribute(transport_kernel_f32<RT_HLL>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4);
    cudaFuncSetAttribute(transport_kernel_f32<RT_GLF>, cudaFuncAttributeMaxDynamicSharedMemorySize, s4);
    cudaFuncSetAttribute(transport_batch_all_kernel<double, RT_HLL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         batch_all_smem<double>());
    cudaFuncSetAttribute(transport_batch_all_kernel<double, RT_GLF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         batch_all_smem<double>());
    cudaFuncSetAttribute(transport_batch_all_kernel<float, RT_HLL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         batch_all_smem<float>());
    cudaFuncSetAttribute(transport_batch_all_kernel<float, RT_GLF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         batch_all_smem<float>());
    set_smem_attr_batch<double, 32, 8>();
    set_smem_attr_batch<double, 16, 16>();
    set_smem_attr_batch<float, 32, 8>();
    set_smem_attr_batch<float, 16, 16>();
}

template <typename S>
static cudaError_t launch_t(const GridDev &g, int G, int flux, double cr, double dt, const S *N0, const S *F0,
                            S *N1, S *F1, const S *tab, const S *inflow, const Partials &p, cudaStream_t st)
{
    const int tiles_x = (g.nx + 31) / 32;
    const int tiles_y = (g.ny + 7) / 8;
    const dim3 grid(p.n_tr_blocks), block(32, 8);
    const size_t smem = sizeof(PlaneSmem<S, 32, 8>);
    const S dtdx = (S)(dt / g.dx);
    const double area_dt = g.dx * g.dx * dt;
    if constexpr (sizeof(S) == sizeof(float)) {
        if (flux == RT_HLL)
            transport_kernel_f32<RT_HLL><<<grid, block, smem, st>>>(g, G, (S)cr, dtdx, area_dt, N0, F0, N1, F1, tab,
                                                                    inflow, p.tr_inbox, p.tr_outflow, tiles_x, tiles_y);
        else
            transport_kernel_f32<RT_GLF><<<grid, block, smem, st>>>(g, G, (S)cr, dtdx, area_dt, N0, F0, N1, F1, tab,
                                                                    inflow, p.tr_inbox, p.tr_outflow, tiles_x, tiles_y);
    } else {
        if (flux == RT_HLL)
            transport_kernel<S, RT_HLL><<<grid, block, smem, st>>>(g, G, (S)cr, dtdx, area_dt, N0, F0, N1, F1, tab,
                                                                   inflow, p.tr_inbox, p.tr_outflow, tiles_x, tiles_y);
        else
            transport_kernel<S, RT_GLF><<<grid, block, smem, st>>>(g, G, (S)cr, dtdx, area_dt, N0, F0, N1, F1, tab,
                                                                   inflow, p.tr_inbox, p.tr_outflow, tiles_x, tiles_y);
    }
    return cudaGetLastError();
}

cudaError_t launch_transport(const GridDev &g, int G, int flux, double cr, double dt,
                             const double *N0, const double *F0, double *N1, double *F1,
                             const double *hll_table, const double *inflow, const Partials &p, cudaStream_t st)
{
    return launch_t<double>(g, G, flux, cr, dt, N0, F0, N1, F1, hll_table, inflow, p, st);
}

cudaError_t launch_transport_f32(const GridDev &g, int G, int flux, double cr, double dt, const float *N0,
                                 const float *F0, float *N1, float *F1, const float *hll_table,
                                 const float *inflow, const Partials &p, cudaStream_t st)
{
    return launch_t<float>(g, G, flux, cr, dt, N0, F0, N1, F1, hll_table, inflow, p, st);
}

template <typename S>
static cudaError_t launch_b(const BatchItem *items, const BatchBox *boxes, int item0, int nitems, int shape,
                            int flux, double cr, double dt, double dx, const void *const *N0, const void *const *F0,
                            void *const *N1, void *const *F1, const S *tab, double *pin, double *pout,
                            cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    S dtdx = (S)(dt / dx);
    double area_dt = dx * dx * dt;
    auto n0 = reinterpret_cast<const S *const *>(N0);
    auto f0 = reinterpret_cast<const S *const *>(F0);
    auto n1 = reinterpret_cast<S *const *>(N1);
    auto f1 = reinterpret_cast<S *const *>(F1);
    if (shape == 0) {
        size_t smem = sizeof(PlaneSmem<S, 32, 8>);
        if (flux == RT_HLL)
            transport_batch_kernel<S, RT_HLL, 32, 8><<<nitems, dim3(32, 8), smem, st>>>(
                items, boxes, (S)cr, dtdx, area_dt, n0, f0, n1, f1, tab, pin, pout, item0);
        else
            transport_batch_kernel<S, RT_GLF, 32, 8><<<nitems, dim3(32, 8), smem, st>>>(
                items, boxes, (S)cr, dtdx, area_dt, n0, f0, n1, f1, tab, pin, pout, item0);
    } else {
        size_t smem = sizeof(PlaneSmem<S, 16, 16>);
        if (flux == RT_HLL)
            transport_batch_kernel<S, RT_HLL, 16, 16><<<nitems, dim3(16, 16), smem, st>>>(
                items, boxes, (S)cr, dtdx, area_dt, n0, f0, n1, f1, tab, pin, pout, item0);
        else
            transport_batch_kernel<S, RT_GLF, 16, 16><<<nitems, dim3(16, 16), smem, st>>>(
                items, boxes, (S)cr, dtdx, area_dt, n0, f0, n1, f1, tab, pin, pout, item0);
    }
    return cudaGetLastError();
}

cudaError_t launch_transport_batch(const BatchItem *items, const BatchBox *boxes, int item0, int nitems,
                                   int shape, bool fp32, int flux, double cr, double dt, double dx,
                                   const void *const *N0, const void *const *F0, void *const *N1,
                                   void *const *F1, const void *tab, double *pin, double *pout, cudaStream_t st)
{
    if (fp32)
        return launch_b<float>(items, boxes, item0, nitems, shape, flux, cr, dt, dx, N0, F0, N1, F1,
                               static_cast<const float *>(tab), pin, pout, st);
    return launch_b<double>(items, boxes, item0, nitems, shape, flux, cr, dt, dx, N0, F0, N1, F1,
                            static_cast<const double *>(tab), pin, pout, st);
}

}  // namespace rtgb

namespace rtgb {

cudaError_t launch_transport_batch_all(const BatchItem *items, const BatchBox *boxes, int n_shape0, int nitems,
                                       bool fp32, int flux, double cr, double dt, double dx, const void *const *N0,
                                       const void *const *F0, void *const *N1, void *const *F1, const void *tab,
                                       double *pin, double *pout, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    const double area_dt = dx * dx * dt;
    if (fp32) {
        using S = float;
        const S dtdx = (S)(dt / dx);
        auto n0 = reinterpret_cast<const S *const *>(N0);
        auto f0 = reinterpret_cast<const S *const *>(F0);
        auto n1 = reinterpret_cast<S *const *>(N1);
        auto f1 = reinterpret_cast<S *const *>(F1);
        const S *t = static_cast<const S *>(tab);
        if (flux == RT_HLL)
            transport_batch_all_kernel<S, RT_HLL><<<nitems, 256, batch_all_smem<S>(), st>>>(
                items, boxes, (S)cr, dtdx, area_dt, n0, f0, n1, f1, t, pin, pout, n_shape0);
        else
            transport_batch_all_kernel<S, RT_GLF><<<nitems, 256, batch_all_smem<S>(), st>>>(
                items, boxes, (S)cr, dtdx, area_dt, n0, f0, n1, f1, t, pin, pout, n_shape0);
    } else {
        using S = double;
        const S dtdx = (S)(dt / dx);
        auto n0 = reinterpret_cast<const S *const *>(N0);
        auto f0 = reinterpret_cast<const S *const *>(F0);
        auto n1 = reinterpret_cast<S *const *>(N1);
        auto f1 = reinterpret_cast<S *const *>(F1);
        const S *t = static_cast<const S *>(tab);
        if (flux == RT_HLL)
            transport_batch_all_kernel<S, RT_HLL><<<nitems, 256, batch_all_smem<S>(), st>>>(
                items, boxes, (S)cr, dtdx, area_dt, n0, f0, n1, f1, t, pin, pout, n_shape0);
        else
            transport_batch_all_kernel<S, RT_GLF><<<nitems, 256, batch_all_smem<S>(), st>>>(
                items, boxes, (S)cr, dtdx, area_dt, n0, f0, n1, f1, t, pin, pout, n_shape0);
    }
    return cudaGetLastError();
}

}  // namespace rtgb

// Adjoint (vector-Jacobian product) of one RT step, FP64, GLF or HLL transport.
//
// The forward step is U_k -> inject -> U_a -> transport -> U_b -> thermo ->
// U_{k+1} (paper Sec. 3: Eq. (injnum), the Godunov update with the GLF
// flux Eq. (glf), the App. A thermochemistry).  Given lambda = dJ/dU_{k+1}
// the reverse sweep is
//   thermo_vjp     lambda_b = (dthermo/dU_b)^T lambda, and dJ/dn_H += ...;
//   transport_vjp  lambda_a = (dtransport/dU_a)^T lambda_b (photons; the
//                  gas passes through unchanged);
//   inject_vjp     dJ/dL_{s,i} += lambda_a(N_i at the source cell) dt / V,
//                  lambda_k = lambda_a.
//
// thermo_vjp differentiates the sub-cycled thermochemistry of one cell in
// forward mode: a team of lanes per cell, lane j seeded with the unit
// tangent of input j (N_0..N_{G-1}, x_HII, x_HeII, x_HeIII, T, n_H), runs
// the thermo_step code of the forward kernels instantiated on dual numbers.
// Its values are the bits of the forward path, so it takes the same
// sub-cycle decisions; the derivative is that of the step sequence the
// forward run took (the schedule is piecewise constant in the inputs).
// Lane j ends with column j of the cell's Jacobian and dots it with lambda.
// The flux output is F' = F prod_s 1/(1 + h_s D_i): its derivative along
// the other inputs enters through w_i = F_i . lambda_{F_i}.
//
// transport_vjp is the transpose of the GLF stencil: with r = dt/dx and
// Phi_d the physical flux along d, every face (L, R) gives U'_L -= r Fhat,
// U'_R += r Fhat with Fhat = (Phi(U_L) + Phi(U_R))/2 - c (U_R - U_L)/2, so
// its co-flux mu = r (lambda'_R - lambda'_L) adds (J_L^T + c) mu/2 to
// lambda_L and (J_R^T - c) mu/2 to lambda_R, J = dPhi_d/dU from the M1
// closure (Sec. 2, Eqs. (edd2), (eddTens)).  Boundary ghosts are B U_c
// (outflow: B = I; reflect: the normal flux negated; inflow: a given state,
// B = 0) and carry no lambda'.
// With HLL (Eq. (hll)) the face flux also depends on the cells' tabulated
// wave speeds; its transpose adds their derivatives (transport_vjp_hll).
// The realisability rescaling of F that ends the forward update is
// transposed first (clamp_vjp); its N < 0 branch (never taken for CFL <= 1)
// is taken as the identity.
#include <cuda_runtime.h>

#include "rt_internal.h"
#include "thermo_step.cuh"

namespace rtgb {
namespace {

using namespace thermo_detail;

constexpr double kClosureFloorN = 1e-30;   // as in the forward closure

// ---------------------------------------------------------------------------
// thermochemistry

template <int G, int GS>
__global__ void __launch_bounds__(128)
thermo_vjp_kernel(ThermoParams p, const double *__restrict__ nH, const double *__restrict__ xHII,
                  const double *__restrict__ xHeII, const double *__restrict__ xHeIII,
                  const double *__restrict__ T, const double *__restrict__ N, const double *__restrict__ F,
                  double *lx, double *ly2, double *ly3, double *lT, const double *__restrict__ lN_in,
                  const double *__restrict__ lF_in, double *__restrict__ lN_out, double *__restrict__ lF_out,
                  double *g_nH, int32_t *sub_out, unsigned *status)
{
    constexpr int NT = G + 5;   // N_i, x_HII, x_HeII, x_HeIII, T, n_H
    static_assert(NT <= GS && 32 % GS == 0, "team size");
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long c = tid / GS;
    const int j = (int)(tid % GS);
    const bool valid = c < p.nc;
    const long long nc = p.nc;

    // every lane reads lambda' before any lane of the warp overwrites it
    double lxv = 0.0, ly2v = 0.0, ly3v = 0.0, lTv = 0.0;
    double lNv[G], w[G];
    if (valid) {
        lxv = lx[c];
        ly2v = ly2[c];
        ly3v = ly3[c];
        lTv = lT[c];
#pragma unroll
        for (int i = 0; i < G; ++i) {
            lNv[i] = lN_in[(long long)i * nc + c];
            const long long b = 3LL * i * nc + c;
            w[i] = F[b] * lF_in[b] + F[b + nc] * lF_in[b + nc] + F[b + 2 * nc] * lF_in[b + 2 * nc];
        }
    }
    __syncwarp();
    if (!valid || j >= NT) return;

    CellState<G, Dual> st;
    st.x = Dual(xHII[c], j == G ? 1.0 : 0.0);
    st.y2 = Dual(xHeII[c], j == G + 1 ? 1.0 : 0.0);
    st.y3 = Dual(xHeIII[c], j == G + 2 ? 1.0 : 0.0);
    st.T = Dual(T[c], j == G + 3 ? 1.0 : 0.0);
#pragma unroll
    for (int i = 0; i < G; ++i) {
        st.N[i] = Dual(N[(long long)i * nc + c], j == i ? 1.0 : 0.0);
        st.Fs[i] = Dual(1.0);
    }
    const Dual n(nH[c], j == G + 4 ? 1.0 : 0.0);
    IsoRates<Dual> iso;
    cell_constants(p, n, iso);
    CoolCache<Dual> cc;
    cc.valid = false;
    cc.rvalid = false;
    if (p.isothermal) {
        RatesT<Dual> t;
        get_rates<false, false>(st.T, p.case_b, kNeedH | (p.helium ? kNeedHe : 0u), kNeedH, t);
        h_rates_from(t, iso.h);
        if (p.helium) he_rates_from(t, iso.he);
    }
    double t_left = p.dt, dt_tc = p.dt;
    int att = 0;
    bool done = false;
    while (!done) {
        done = subcycle_once<G, false, false, Dual>(p, n, st, t_left, dt_tc, att, iso, cc);
        if (!done && att >= p.max_sub) {
            atomicOr(status, kStatusSubcycle);
            done = true;
        }
    }

    double g = lxv * st.x.d + ly2v * st.y2.d + ly3v * st.y3.d + lTv * st.T.d;
#pragma unroll
    for (int i = 0; i < G; ++i) g += lNv[i] * st.N[i].d + w[i] * st.Fs[i].d;
    if (!isfinite(g)) atomicOr(status, kStatusNonFinite);

    if (j < G) {
        lN_out[(long long)j * nc + c] = g;
    } else if (j == G) {
        lx[c] = g;
    } else if (j == G + 1) {
        ly2[c] = g;
    } else if (j == G + 2) {
        ly3[c] = g;
    } else if (j == G + 3) {
        lT[c] = g;
    } else {
        g_nH[c] += g;
    }
    if (j == 0) {
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const long long b = 3LL * i * nc + c;
            const double s = st.Fs[i].v;
            lF_out[b] = s * lF_in[b];
            lF_out[b + nc] = s * lF_in[b + nc];
            lF_out[b + 2 * nc] = s * lF_in[b + 2 * nc];
        }
        if (sub_out) sub_out[c] = att;
    }
}

template <int G>
cudaError_t launch_thermo_vjp_g(const ThermoParams &tp, const double *nH, const double *xHII, const double *xHeII,
                                const double *xHeIII, const double *T, const double *N, const double *F, double *lx,
                                double *ly2, double *ly3, double *lT, const double *lN_in, const double *lF_in,
                                double *lN_out, double *lF_out, double *g_nH, int32_t *sub_out, unsigned *status,
                                cudaStream_t s)
{
    constexpr int GS = (G + 5 <= 8) ? 8 : 16;
    const long long threads = tp.nc * GS;
    const long long blocks = (threads + 127) / 128;
    thermo_vjp_kernel<G, GS><<<(unsigned)blocks, 128, 0, s>>>(tp, nH, xHII, xHeII, xHeIII, T, N, F, lx, ly2, ly3, lT,
                                                               lN_in, lF_in, lN_out, lF_out, g_nH, sub_out, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// transport

// v^T dPhi_d/dU at U = (N, F): the gradient of s(U) = v_N F_d + v_F . P e_d
// with P = c^2 N (a I + b n n^T), a = (1 - chi)/2, b = (3 chi - 1)/2,
// f = |F|/(c N), n = F/|F|.  With f' = df/dN = -f/N, df/dF = n/(c N),
// dn/dF = (I - n n^T)/|F|:
//   ds/dN = c^2 (a v_d + b (v.n) n_d) - c^2 f (a' v_d + b' (v.n) n_d)
//   ds/dF = v_N e_d + c (a' v_d + b' (v.n) n_d) n
//           + (c^2 N b / |F|) (n_d (v - (v.n) n) + (v.n)(e_d - n_d n))
// (v is the flux part of v here).  f is clamped to 1 in the closure, so
// where the clamp acts the terms through df vanish; below the N floor or at
// F = 0 the closure is isotropic (f = 0, a = 1/3, b = 0).
// b is taken in a form free of cancellation: with q = sqrt(4 - 3 f^2),
// 3 chi - 1 = f^2 (6/(2 + q) + 12)/(5 + 2 q), so b = f^2 B(f) with
// B = (3/(2 + q) + 6)/(5 + 2 q), and c^2 N b / |F| = c f B.  Written as
// 0.5 (3 chi - 1), b is rounding noise of ~1e-17 for f << 1e-8, and that
// noise divided by |F| = c N f grew without bound as f -> 0.
__device__ __forceinline__ void phi_vjp(double N, const double F[3], int d, double c, const double v[4],
                                        double out[4])
{
    const double F2 = F[0] * F[0] + F[1] * F[1] + F[2] * F[2];
    double f = 0.0, n[3] = {0.0, 0.0, 0.0}, mag = 0.0;
    bool clamped = false, dir = false;
    if (N > kClosureFloorN && F2 > 0.0) {
        mag = sqrt(F2);
        const double fr = mag / (c * N);
        clamped = fr > 1.0;
        f = clamped ? 1.0 : fr;
        n[0] = F[0] / mag; n[1] = F[1] / mag; n[2] = F[2] / mag;
        dir = true;
    }
    const double f2 = f * f;
    const double q = sqrt(4.0 - 3.0 * f2);
    const double den = 5.0 + 2.0 * q;
    const double chi = (3.0 + 4.0 * f2) / den;
    const double dchi = (8.0 * f * den + 6.0 * f * (3.0 + 4.0 * f2) / q) / (den * den);
    const double B = (3.0 / (2.0 + q) + 6.0) / den;
    const double a = 0.5 * (1.0 - chi), b = f2 * B;
    const double da = -0.5 * dchi, db = 1.5 * dchi;
    const double vn = v[1] * n[0] + v[2] * n[1] + v[3] * n[2];
    const double vd = v[1 + d], nd = n[d];
    const double c2 = c * c;
    double gN = c2 * (a * vd + b * vn * nd);
    if (!clamped) gN -= c2 * f * (da * vd + db * vn * nd);
    out[0] = gN;
    out[1] = out[2] = out[3] = 0.0;
    out[1 + d] = v[0];
    if (dir) {
        const double k1 = clamped ? 0.0 : c * (da * vd + db * vn * nd);
        // c^2 N b / |F| = c b / (|F| / (c N)): c f B unclamped; clamped
        // (f = 1 < |F| / (c N)), c b(1) c N / |F|
        const double K = clamped ? c * b * (c * N / mag) : c * f * B;
#pragma unroll
        for (int k = 0; k < 3; ++k)
            out[1 + k] += k1 * n[k] + K * (nd * (v[1 + k] - vn * n[k]) + vn * ((k == d ? 1.0 : 0.0) - nd * n[k]));
    }
}

__global__ void __launch_bounds__(128)
transport_vjp_kernel(GridDev g, double c, double r, const double *__restrict__ N, const double *__restrict__ F,
                     const double *__restrict__ lN1, const double *__restrict__ lF1, double *__restrict__ lN0,
                     double *__restrict__ lF0)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nc) return;
    const long long go = (long long)blockIdx.y * g.stride;   // group offset of N and lambda_N
    const double *Ng = N + go, *Fg = F + 3 * go, *lNg = lN1 + go, *lFg = lF1 + 3 * go;
    const int x = (int)(i % g.nx);
    const int y = (int)((i / g.nx) % g.ny);
    const int z = (int)(i / ((long long)g.nx * g.ny));
    const int pos[3] = {x, y, z};
    const int ext[3] = {g.nx, g.ny, g.nz};
    const long long step[3] = {1, g.nx, (long long)g.nx * g.ny};

    const double Nc = Ng[i];
    const double Fc[3] = {Fg[i], Fg[g.stride + i], Fg[2 * g.stride + i]};
    double lp[4] = {lNg[i], lFg[i], lFg[g.stride + i], lFg[2 * g.stride + i]};
    double acc[4] = {lp[0], lp[1], lp[2], lp[3]};

#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double m[4] = {0.0, 0.0, 0.0, 0.0};   // times J_c^T
#pragma unroll
        for (int side = 0; side < 2; ++side) {   // 0: low face, 1: high face
            const int bcode = g.bc[2 * d + side];
            const bool at_edge = side ? (pos[d] == ext[d] - 1) : (pos[d] == 0);
            double mu[4];
            if (!at_edge || bcode == RT_BC_PERIODIC) {
                long long nb;
                if (!at_edge) nb = side ? i + step[d] : i - step[d];
                else nb = side ? i - (long long)(ext[d] - 1) * step[d] : i + (long long)(ext[d] - 1) * step[d];
                const double ln[4] = {lNg[nb], lFg[nb], lFg[g.stride + nb], lFg[2 * g.stride + nb]};
#pragma unroll
                for (int k = 0; k < 4; ++k) mu[k] = side ? r * (ln[k] - lp[k]) : r * (lp[k] - ln[k]);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    m[k] += 0.5 * mu[k];
                    acc[k] += side ? 0.5 * c * mu[k] : -0.5 * c * mu[k];
                }
            } else {
                // ghost B U_c: high face mu = -r lambda'_c, low face mu = r lambda'_c
#pragma unroll
                for (int k = 0; k < 4; ++k) mu[k] = side ? -r * lp[k] : r * lp[k];
                // this cell's own side of the face
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    m[k] += 0.5 * mu[k];
                    acc[k] += side ? 0.5 * c * mu[k] : -0.5 * c * mu[k];
                }
                if (bcode == RT_BC_INFLOW) continue;   // a given ghost state: B = 0
                // the ghost's side, through B (B^T = B)
                const double sgn = side ? -0.5 * c : 0.5 * c;
                if (bcode == RT_BC_REFLECT) {
                    double Fgh[3] = {Fc[0], Fc[1], Fc[2]};
                    Fgh[d] = -Fgh[d];
                    double jg[4];
                    phi_vjp(Nc, Fgh, d, c, mu, jg);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        double t = 0.5 * jg[k] + sgn * mu[k];
                        acc[k] += (k == 1 + d) ? -t : t;
                    }
                } else {   // outflow: B = I, J_ghost = J_c
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        m[k] += 0.5 * mu[k];
                        acc[k] += sgn * mu[k];
                    }
                }
            }
        }
        double jm[4];
        phi_vjp(Nc, Fc, d, c, m, jm);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += jm[k];
    }
    double *lNo = lN0 + go, *lFo = lF0 + 3 * go;
    lNo[i] = acc[0];
    lFo[i] = acc[1];
    lFo[g.stride + i] = acc[2];
    lFo[2 * g.stride + i] = acc[3];
}

// ---- HLL (Eq. (hll)) ----
//
// Face flux Fhat = (l+ Phi_L - l- Phi_R + l+ l- (U_R - U_L)) / (l+ - l-),
// l+ = max(0, lmax_L, lmax_R), l- = min(0, lmin_L, lmin_R), the speeds c
// times the bilinear table at (f, mu_d) of their cell.  Its transpose on a
// co-flux m: (l+ J_L^T m - l+ l- m)/den to U_L, (-l- J_R^T m + l+ l- m)/den
// to U_R, and through the speeds: d(Fhat.m)/dl+ = (Phi_L + l- dU - Fhat).m
// / den, d(Fhat.m)/dl- = (-Phi_R + l+ dU + Fhat).m / den, times the
// gradient of the selected cell's speed (the max/min picks one cell; the
// bilinear table is differentiated inside its cell).  With no speed (both
// zero: f = 1 beams along the face) the flux is the average of the two.

struct HllSide {
    double U[4], Phi[4];
    double lo, hi;            // c * table speeds
    double dlo[4], dhi[4];    // their gradients with respect to U
};

// speeds and their U-gradients of a state along direction d
__device__ __forceinline__ void hll_side(const double U[4], int d, double c, const double *__restrict__ tab, HllSide &o)
{
    const double N = U[0];
    const double F2 = U[1] * U[1] + U[2] * U[2] + U[3] * U[3];
    double f = 0.0, n[3] = {0.0, 0.0, 0.0}, mag = 0.0;
    bool dir = false, clamped = false;
    if (N > kClosureFloorN && F2 > 0.0) {
        mag = sqrt(F2);
        const double fr = mag / (c * N);
        clamped = fr > 1.0;
        f = clamped ? 1.0 : fr;
        n[0] = U[1] / mag; n[1] = U[2] / mag; n[2] = U[3] / mag;
        dir = true;
    }
    const double mu = n[d];
    // the forward's bilinear lookup, with its slopes
    const double fx = f * (double)(kHllNF - 1);
    int k = (int)floor(fx);
    k = k < 0 ? 0 : (k > kHllNF - 2 ? kHllNF - 2 : k);
    const double wf = fx - (double)k;
    const double mx = (mu + 1.0) * 0.5 * (double)(kHllNMU - 1);
    int j = (int)floor(mx);
    j = j < 0 ? 0 : (j > kHllNMU - 2 ? kHllNMU - 2 : j);
    const double wm = mx - (double)j;
    const double2 *t2 = reinterpret_cast<const double2 *>(tab);
    const double2 A = __ldg(&t2[k * kHllNMU + j]), B = __ldg(&t2[k * kHllNMU + j + 1]);
    const double2 Cc = __ldg(&t2[(k + 1) * kHllNMU + j]), D = __ldg(&t2[(k + 1) * kHllNMU + j + 1]);
    const double lo0 = A.x + wm * (B.x - A.x), lo1 = Cc.x + wm * (D.x - Cc.x);
    const double hi0 = A.y + wm * (B.y - A.y), hi1 = Cc.y + wm * (D.y - Cc.y);
    o.lo = (lo0 + wf * (lo1 - lo0)) * c;
    o.hi = (hi0 + wf * (hi1 - hi0)) * c;
    // d/df and d/dmu of the table values, times c
    const double sf = (double)(kHllNF - 1) * c, sm = 0.5 * (double)(kHllNMU - 1) * c;
    const double dlo_df = sf * (lo1 - lo0), dhi_df = sf * (hi1 - hi0);
    const double dlo_dmu = sm * ((1.0 - wf) * (B.x - A.x) + wf * (D.x - Cc.x));
    const double dhi_dmu = sm * ((1.0 - wf) * (B.y - A.y) + wf * (D.y - Cc.y));
    for (int q = 0; q < 4; ++q) o.dlo[q] = o.dhi[q] = 0.0;
    if (dir) {
        // f = |F|/(c N): df/dN = -f/N, df/dF = n/(c N) (0 where clamped);
        // mu = F_d/|F|: dmu/dF = (e_d - mu n)/|F|
        const double dfN = clamped ? 0.0 : -f / N;
        const double dfF = clamped ? 0.0 : 1.0 / (c * N);
        o.dlo[0] = dlo_df * dfN;
        o.dhi[0] = dhi_df * dfN;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double dmu = ((q == d ? 1.0 : 0.0) - mu * n[q]) / mag;
            o.dlo[1 + q] = dlo_df * dfF * n[q] + dlo_dmu * dmu;
            o.dhi[1 + q] = dhi_df * dfF * n[q] + dhi_dmu * dmu;
        }
    }
    // physical flux along d
    double Fv[3] = {U[1], U[2], U[3]};
    double P[3];
    {
        const double f2 = f * f;
        const double chi = (3.0 + 4.0 * f2) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f2));
        const double cN = c * c * N;
        const double ca = cN * 0.5 * (1.0 - chi), cb = cN * 0.5 * (3.0 * chi - 1.0);
#pragma unroll
        for (int q = 0; q < 3; ++q) P[q] = (q == d ? ca : 0.0) + cb * n[q] * n[d];
    }
    o.Phi[0] = Fv[d];
    o.Phi[1] = P[0]; o.Phi[2] = P[1]; o.Phi[3] = P[2];
#pragma unroll
    for (int q = 0; q < 4; ++q) o.U[q] = U[q];
}

// Contribution of one HLL face (L, R) with co-flux m to the lambda of L
// (want_L) and / or R; JLm, JRm: J_L^T m and J_R^T m where needed.
__device__ __forceinline__ void hll_face_vjp(const HllSide &L, const HllSide &R, const double m[4],
                                             const double JLm[4], const double JRm[4], bool want_L, bool want_R,
                                             double cL[4], double cR[4])
{
    const double lp = fmax(0.0, fmax(L.hi, R.hi));
    const double lm = fmin(0.0, fmin(L.lo, R.lo));
    const double den = lp - lm;
    if (!(den > 0.0)) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            cL[q] = want_L ? 0.5 * JLm[q] : 0.0;
            cR[q] = want_R ? 0.5 * JRm[q] : 0.0;
        }
        return;
    }
    const double inv = 1.0 / den;
    double gp = 0.0, gm = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double dU = R.U[q] - L.U[q];
        const double Fh = (lp * L.Phi[q] - lm * R.Phi[q] + lp * lm * dU) * inv;
        gp += (L.Phi[q] + lm * dU - Fh) * m[q];
        gm += (-R.Phi[q] + lp * dU + Fh) * m[q];
    }
    gp *= inv;
    gm *= inv;
    // which cell's speed sets l+ and l- (none if the bound is 0)
    const bool pL = lp > 0.0 && L.hi >= R.hi, pR = lp > 0.0 && !pL;
    const bool mL = lm < 0.0 && L.lo <= R.lo, mR = lm < 0.0 && !mL;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        cL[q] = want_L ? (lp * JLm[q] - lp * lm * m[q]) * inv + (pL ? gp * L.dhi[q] : 0.0) + (mL ? gm * L.dlo[q] : 0.0)
                       : 0.0;
        cR[q] = want_R ? (-lm * JRm[q] + lp * lm * m[q]) * inv + (pR ? gp * R.dhi[q] : 0.0) + (mR ? gm * R.dlo[q] : 0.0)
                       : 0.0;
    }
}

__global__ void __launch_bounds__(128)
transport_vjp_hll_kernel(GridDev g, double c, double r, const double *__restrict__ N, const double *__restrict__ F,
                         const double *__restrict__ tab, const double *__restrict__ inflow,
                         const double *__restrict__ lN1,
                         const double *__restrict__ lF1, double *__restrict__ lN0, double *__restrict__ lF0)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.nc) return;
    const long long go = (long long)blockIdx.y * g.stride;
    const double *Ng = N + go, *Fg = F + 3 * go, *lNg = lN1 + go, *lFg = lF1 + 3 * go;
    const int x = (int)(i % g.nx);
    const int y = (int)((i / g.nx) % g.ny);
    const int z = (int)(i / ((long long)g.nx * g.ny));
    const int pos[3] = {x, y, z};
    const int ext[3] = {g.nx, g.ny, g.nz};
    const long long step[3] = {1, g.nx, (long long)g.nx * g.ny};
    const double Uc[4] = {Ng[i], Fg[i], Fg[g.stride + i], Fg[2 * g.stride + i]};
    const double lp[4] = {lNg[i], lFg[i], lFg[g.stride + i], lFg[2 * g.stride + i]};
    double acc[4] = {lp[0], lp[1], lp[2], lp[3]};
    const double zero[4] = {0.0, 0.0, 0.0, 0.0};

#pragma unroll 1
    for (int d = 0; d < 3; ++d) {
        HllSide S;
        hll_side(Uc, d, c, tab, S);
#pragma unroll 1
        for (int side = 0; side < 2; ++side) {   // 0: low face (c is R), 1: high face (c is L)
            const int bcode = g.bc[2 * d + side];
            const bool at_edge = side ? (pos[d] == ext[d] - 1) : (pos[d] == 0);
            double m[4], Jc[4], cL[4], cR[4];
            if (!at_edge || bcode == RT_BC_PERIODIC) {
                long long nb;
                if (!at_edge) nb = side ? i + step[d] : i - step[d];
                else nb = side ? i - (long long)(ext[d] - 1) * step[d] : i + (long long)(ext[d] - 1) * step[d];
                const double Un[4] = {Ng[nb], Fg[nb], Fg[g.stride + nb], Fg[2 * g.stride + nb]};
                const double ln[4] = {lNg[nb], lFg[nb], lFg[g.stride + nb], lFg[2 * g.stride + nb]};
                HllSide Sn;
                hll_side(Un, d, c, tab, Sn);
#pragma unroll
                for (int q = 0; q < 4; ++q) m[q] = side ? r * (ln[q] - lp[q]) : r * (lp[q] - ln[q]);
                phi_vjp(Uc[0], Uc + 1, d, c, m, Jc);
                if (side) hll_face_vjp(S, Sn, m, Jc, zero, true, false, cL, cR);
                else hll_face_vjp(Sn, S, m, zero, Jc, false, true, cL, cR);
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] += side ? cL[q] : cR[q];
            } else {
                // ghost B U_c (outflow: B = I; reflect: normal flux negated);
                // it carries no lambda', and its side reaches c through B
                double Ug[4] = {Uc[0], Uc[1], Uc[2], Uc[3]};
                if (bcode == RT_BC_REFLECT) Ug[1 + d] = -Ug[1 + d];
                const bool fixed = bcode == RT_BC_INFLOW;   // a given ghost state: B = 0
                if (fixed) {
                    const int face = 2 * d + side;
#pragma unroll
                    for (int q = 0; q < 4; ++q) Ug[q] = inflow ? inflow[24 * blockIdx.y + 4 * face + q] : 0.0;
                }
                HllSide Sg;
                hll_side(Ug, d, c, tab, Sg);
#pragma unroll
                for (int q = 0; q < 4; ++q) m[q] = side ? -r * lp[q] : r * lp[q];
                double Jg[4];
                phi_vjp(Uc[0], Uc + 1, d, c, m, Jc);
                phi_vjp(Ug[0], Ug + 1, d, c, m, Jg);
                if (side) hll_face_vjp(S, Sg, m, Jc, Jg, true, true, cL, cR);
                else hll_face_vjp(Sg, S, m, Jg, Jc, true, true, cL, cR);
                const double *self = side ? cL : cR, *gh = side ? cR : cL;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double gq = fixed ? 0.0 : ((bcode == RT_BC_REFLECT && q == 1 + d) ? -gh[q] : gh[q]);
                    acc[q] += self[q] + gq;
                }
            }
        }
    }
    double *lNo = lN0 + go, *lFo = lF0 + 3 * go;
    lNo[i] = acc[0];
    lFo[i] = acc[1];
    lFo[g.stride + i] = acc[2];
    lFo[2 * g.stride + i] = acc[3];
}

// The forward update ends by rescaling F to c N where |F| came out above it
// (rounding level for CFL <= 1, but it does happen where HLL keeps beams at
// f = 1).  Its output is then exactly on |F| = c N, which is where it is
// recognised here (|F|^2 >= (c N)^2 (1 - 1e-12)); the map F -> c N F/|F|
// has the transpose lambda_N += c n.lambda_F, lambda_F -> (I - n n^T)
// lambda_F, applied in place before the flux transpose.
__global__ void clamp_vjp_kernel(long long n, double c, const double *__restrict__ N, const double *__restrict__ F,
                                 double *lN, double *lF, long long nc)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // over G * nc
    if (k >= n) return;
    const long long g = k / nc, i = k % nc;
    const double Nv = N[k];
    const long long b = 3 * g * nc + i;
    const double f0 = F[b], f1 = F[b + nc], f2 = F[b + 2 * nc];
    const double F2 = f0 * f0 + f1 * f1 + f2 * f2;
    const double cn = c * Nv;
    if (!(Nv > kClosureFloorN) || !(F2 >= cn * cn * (1.0 - 1e-12))) return;
    const double mag = sqrt(F2);
    const double n0 = f0 / mag, n1 = f1 / mag, n2 = f2 / mag;
    const double l0 = lF[b], l1 = lF[b + nc], l2 = lF[b + 2 * nc];
    const double nl = n0 * l0 + n1 * l1 + n2 * l2;
    lN[k] += c * nl;
    lF[b] = l0 - n0 * nl;
    lF[b + nc] = l1 - n1 * nl;
    lF[b + 2 * nc] = l2 - n2 * nl;
}

// dJ/dL_{s,i} += lambda_a(N_i at the cell of source s) dt / V
__global__ void inject_vjp_kernel(int nsrc, int G, long long nc, const long long *__restrict__ cells,
                                  const double *__restrict__ lN, double dt_over_V, double *g_L)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsrc) return;
    const long long c = cells[s];
    for (int k = 0; k < G; ++k) g_L[(long long)s * G + k] += lN[(long long)k * nc + c] * dt_over_V;
}

__global__ void count_mismatch_kernel(long long n, const int32_t *__restrict__ a, const int32_t *__restrict__ b,
                                      unsigned long long *count)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool m = i < n && a[i] != b[i];
    const unsigned ball = __ballot_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && ball) atomicAdd(count, (unsigned long long)__popc(ball));
}

}  // namespace

cudaError_t launch_thermo_vjp(const ThermoParams &tp, int G, const double *nH, const double *xHII,
                              const double *xHeII, const double *xHeIII, const double *T, const double *N,
                              const double *F, double *lx, double *ly2, double *ly3, double *lT,
                              const double *lN_in, const double *lF_in, double *lN_out, double *lF_out,
                              double *g_nH, int32_t *sub_out, unsigned *status, cudaStream_t s)
{
#define RTGB_TVJP(GG)                                                                                             \
    case GG:                                                                                                      \
        return launch_thermo_vjp_g<GG>(tp, nH, xHII, xHeII, xHeIII, T, N, F, lx, ly2, ly3, lT, lN_in, lF_in, lN_out, \
                                       lF_out, g_nH, sub_out, status, s);
    switch (G) {
        RTGB_TVJP(1)
        RTGB_TVJP(2)
        RTGB_TVJP(3)
        RTGB_TVJP(4)
        RTGB_TVJP(5)
        RTGB_TVJP(6)
        RTGB_TVJP(7)
        RTGB_TVJP(8)
    default: return cudaErrorInvalidValue;
    }
#undef RTGB_TVJP
}

cudaError_t launch_transport_vjp(const GridDev &g, int G, int flux, double cr, double dt, const double *N,
                                 const double *F, const double *hll_table, const double *inflow,
                                 const double *lN1, const double *lF1, double *lN0, double *lF0, cudaStream_t s)
{
    dim3 grid((unsigned)((g.nc + 127) / 128), (unsigned)G);
    if (flux == RT_HLL)
        transport_vjp_hll_kernel<<<grid, 128, 0, s>>>(g, cr, dt / g.dx, N, F, hll_table, inflow, lN1, lF1, lN0,
                                                      lF0);
    else
        transport_vjp_kernel<<<grid, 128, 0, s>>>(g, cr, dt / g.dx, N, F, lN1, lF1, lN0, lF0);
    return cudaGetLastError();
}

cudaError_t launch_clamp_vjp(int G, long long nc, double cr, const double *N, const double *F, double *lN, double *lF,
                             cudaStream_t s)
{
    const long long n = (long long)G * nc;
    clamp_vjp_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, cr, N, F, lN, lF, nc);
    return cudaGetLastError();
}

cudaError_t launch_inject_vjp(int nsrc, int G, long long nc, const long long *cells, const double *lN,
                              double dt_over_V, double *g_L, cudaStream_t s)
{
    if (nsrc <= 0) return cudaSuccess;
    inject_vjp_kernel<<<(nsrc + 127) / 128, 128, 0, s>>>(nsrc, G, nc, cells, lN, dt_over_V, g_L);
    return cudaGetLastError();
}

cudaError_t launch_count_mismatch(long long n, const int32_t *a, const int32_t *b, unsigned long long *count,
                                  cudaStream_t s)
{
    count_mismatch_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, b, count);
    return cudaGetLastError();
}

}  // namespace rtgb

// Host-side table of the HLL wave speeds (paper Sec. 3.2, Eq. (hll)).
//
// The HLL flux needs lambda_min / lambda_max, the extreme eigenvalues of the
// Jacobian dF/dU of the M1 system, which depend only on the reduced flux f
// and the cosine mu between the flux direction and the face normal.  The
// paper reads them from a table of Gonzalez et al. (2007) that it does not
// print; here they are computed in closed form (in units of c):
//
// For the x-direction flux [F_x, P_xx, P_xy, P_xz], P = N D(f, n) with the
// Eddington tensor D = a I + b n n^T, a = (1-chi)/2, b = (3 chi - 1)/2
// (Eqs. (eddTens), (Udir)), and n = (mu, sqrt(1-mu^2), 0), the Jacobian at
// N = 1 is
//     dF_x/dN        = 1 (column 1 of row 0)
//     dP_xj/dN       = d_xj (a - f a') + n_x n_j (b - f b')
//     dP_xj/dF_k     = d_xj a' n_k + b' n_x n_j n_k + (b/f)(d_xk n_j + d_jk n_x - 2 n_x n_j n_k)
// with a' = -chi'/2, b' = 3 chi'/2.  Its characteristic polynomial has the
// factor (lambda - mu b/f) twice (the two transverse modes); dividing the
// cubic of the (N, F_x, F_y) block by that root leaves a quadratic whose two
// roots are the longitudinal speeds.  The extremes are taken over all four.
// At f = 0 the speeds are -1/sqrt(3), +1/sqrt(3); at f = 1 all four
// coalesce onto mu, which is stored exactly.
#include <cmath>
#include <cstddef>

namespace rtgb {

static void chi_and_derivative(double f, double *chi, double *dchi)
{
    double S = std::sqrt(4.0 - 3.0 * f * f);
    double den = 5.0 + 2.0 * S;
    *chi = (3.0 + 4.0 * f * f) / den;
    *dchi = (8.0 * f * den + (3.0 + 4.0 * f * f) * 6.0 * f / S) / (den * den);
}

void hll_speeds(double f, double mu, double *lmin, double *lmax)
{
    if (f <= 0.0) {
        double r = 1.0 / std::sqrt(3.0);
        *lmin = -r;
        *lmax = r;
        return;
    }
    if (f >= 1.0) {
        *lmin = mu;
        *lmax = mu;
        return;
    }
    double chi, dchi;
    chi_and_derivative(f, &chi, &dchi);
    const double a = 0.5 * (1.0 - chi), b = 0.5 * (3.0 * chi - 1.0);
    const double ap = -0.5 * dchi, bp = 1.5 * dchi;
    const double n[3] = {mu, std::sqrt(std::fmax(0.0, 1.0 - mu * mu)), 0.0};
    // 3x3 block over (N, F_x, F_y); the F_z column/row decouples.
    double M[3][3];
    M[0][0] = 0.0; M[0][1] = 1.0; M[0][2] = 0.0;
    for (int j = 0; j < 2; ++j) {             // rows P_xx, P_xy
        double dxj = (j == 0) ? 1.0 : 0.0;
        M[1 + j][0] = dxj * (a - f * ap) + n[0] * n[j] * (b - f * bp);
        for (int k = 0; k < 2; ++k) {
            double dxk = (k == 0) ? 1.0 : 0.0;
            double djk = (j == k) ? 1.0 : 0.0;
            M[1 + j][1 + k] = dxj * ap * n[k] + bp * n[0] * n[j] * n[k]
                              + (b / f) * (dxk * n[j] + djk * n[0] - 2.0 * n[0] * n[j] * n[k]);
        }
    }
    // characteristic polynomial lambda^3 + c2 lambda^2 + c1 lambda + c0
    double tr = M[0][0] + M[1][1] + M[2][2];
    double minors = (M[0][0] * M[1][1] - M[0][1] * M[1][0]) + (M[0][0] * M[2][2] - M[0][2] * M[2][0])
                    + (M[1][1] * M[2][2] - M[1][2] * M[2][1]);
    double c2 = -tr, c1 = minors;
    double r = mu * b / f;                     // transverse speed (double root)
    // deflate: (lambda - r)(lambda^2 + p1 lambda + p0)
    double p1 = c2 + r;
    double p0 = c1 + r * p1;
    double disc = p1 * p1 - 4.0 * p0;
    if (disc < 0.0) disc = 0.0;
    double sq = std::sqrt(disc);
    // numerically stable pair of roots
    double q = -0.5 * (p1 + (p1 >= 0.0 ? sq : -sq));
    double r1 = q;
    double r2 = (q != 0.0) ? p0 / q : 0.0;
    double lo = std::fmin(std::fmin(r1, r2), r);
    double hi = std::fmax(std::fmax(r1, r2), r);
    *lmin = lo;
    *lmax = hi;
}

void hll_table(int nf, int nmu, double *out)
{
    for (int k = 0; k < nf; ++k) {
        double f = (double)k / (double)(nf - 1);
        for (int j = 0; j < nmu; ++j) {
            double mu = -1.0 + 2.0 * (double)j / (double)(nmu - 1);
            double lo, hi;
            hll_speeds(f, mu, &lo, &hi);
            out[((size_t)k * nmu + j) * 2 + 0] = lo;
            out[((size_t)k * nmu + j) * 2 + 1] = hi;
        }
    }
}

}  // namespace rtgb

// Device rate-coefficient fits of the paper's appendix on interaction rate
// coefficients (collisional ionisation: Cen 1992; recombination and
// recombination cooling: Hui & Gnedin 1997; collisional excitation: Cen
// 1992; bremsstrahlung; Compton: Haiman et al. 1996; dielectronic: Black
// 1981), each with its analytic temperature derivative, in FP64.
//
// Transcendentals are shared: ln T, sqrt T and 1/T once per temperature;
// each Boltzmann factor exp(-T0/T) serves both the collisional ionisation
// rate and its cooling rate; every Hui & Gnedin form
// A lam^p / (1 + (lam/l0)^r)^s is one log1p and two exp.
#pragma once

#include <cuda_runtime.h>

namespace rtgb {

struct TVars {
    double T, invT, lnT, sqrtT, u;   // u = 1 / (1 + sqrt(T / 1e5))
};

__device__ __forceinline__ TVars tvars(double T)
{
    TVars v;
    v.T = T;
    v.invT = 1.0 / T;
    v.lnT = log(T);
    v.sqrtT = sqrt(T);
    v.u = 1.0 / (1.0 + v.sqrtT * 0.003162277660168379);
    return v;
}

// A sqrt(T) u exp(-T0/T), given e = exp(-T0/T)
__device__ __forceinline__ void cen_fit(double A, double T0, double e, const TVars &t, double &v, double &dv)
{
    v = A * t.sqrtT * t.u * e;
    dv = v * (0.5 * t.u * t.invT + T0 * t.invT * t.invT);
}

// A lam^p / (1 + (lam/l0)^r)^s, lam = T1 / T; lnT1 = ln T1, lnl0 = ln l0
__device__ __forceinline__ void hg_fit(double A, double lnT1, double p, double lnl0, double r, double s,
                                       const TVars &t, double &v, double &dv)
{
    double lnlam = lnT1 - t.lnT;
    double w = exp(r * (lnlam - lnl0));
    double l1w = log1p(w);
    v = A * exp(p * lnlam - s * l1w);
    dv = -v * t.invT * (p - s * r * w / (1.0 + w));
}

// A lam^p, lam = T1 / T
__device__ __forceinline__ void pow_fit(double A, double lnT1, double p, const TVars &t, double &v, double &dv)
{
    v = A * exp(p * (lnT1 - t.lnT));
    dv = -v * p * t.invT;
}

// ln of the fit temperatures and pivots
#define RTGB_LN_315614 12.662275226919286     // HI
#define RTGB_LN_570670 13.254566388120152     // HeI
#define RTGB_LN_1263030 14.049024154019651    // HeII
#define RTGB_LN_2_74 1.007957920399979
#define RTGB_LN_0_522 -0.6500876910994983
#define RTGB_LN_2_25 0.8109302162163288
#define RTGB_LN_0_541 -0.6143360001356555

struct HRates {       // rates needed by the x_HII update
    double beta, dbeta, alpha, dalpha;
};

__device__ __forceinline__ void h_rates(const TVars &t, int case_b, HRates &r)
{
    cen_fit(5.85e-11, 157809.1, exp(-157809.1 * t.invT), t, r.beta, r.dbeta);
    if (case_b)
        hg_fit(2.753e-14, RTGB_LN_315614, 1.5, RTGB_LN_2_74, 0.407, 2.242, t, r.alpha, r.dalpha);
    else
        hg_fit(1.269e-13, RTGB_LN_315614, 1.503, RTGB_LN_0_522, 0.47, 1.923, t, r.alpha, r.dalpha);
}

struct HeRates {
    double beta_HeI, beta_HeII, alpha_HeII, alpha_HeIII;
};

__device__ __forceinline__ void he_rates(const TVars &t, int case_b, bool need_hei, HeRates &r)
{
    double d;
    if (need_hei) {
        cen_fit(2.38e-11, 285335.4, exp(-285335.4 * t.invT), t, r.beta_HeI, d);
        if (case_b) pow_fit(1.26e-14, RTGB_LN_570670, 0.75, t, r.alpha_HeII, d);
        else pow_fit(3e-14, RTGB_LN_570670, 0.654, t, r.alpha_HeII, d);
    }
    cen_fit(5.68e-12, 631515.0, exp(-631515.0 * t.invT), t, r.beta_HeII, d);
    if (case_b)
        hg_fit(5.506e-14, RTGB_LN_1263030, 1.5, RTGB_LN_2_74, 0.407, 2.242, t, r.alpha_HeIII, d);
    else
        hg_fit(2.538e-13, RTGB_LN_1263030, 1.503, RTGB_LN_0_522, 0.47, 1.923, t, r.alpha_HeIII, d);
}

// Primordial cooling magnitude L (Eq. (rate_cooling), positive = cooling)
// and dL/dT, for the given absorber/ion densities and electron density.
__device__ __forceinline__ void cooling(const TVars &t, int case_b, double a_exp, bool helium, double ne,
                                        double nHI, double nHII, double nHeI, double nHeII, double nHeIII,
                                        double &L, double &dL)
{
    const double kB = 1.380649e-16;
    double v, dv;
    double e1 = exp(-157809.1 * t.invT);
    double e4 = exp(-118348.0 * t.invT);
    // zeta_HI + psi_HI on n_e n_HI
    cen_fit(1.27e-21, 157809.1, e1, t, v, dv);
    double psi = 7.5e-19 * t.u * e4;
    double dpsi = psi * (-0.5 * (1.0 - t.u) * t.invT + 118348.0 * t.invT * t.invT);
    double Ls = (v + psi) * nHI;
    double dLs = (dv + dpsi) * nHI;
    // recombination cooling eta_HII T-form
    double eta, deta;
    if (case_b) hg_fit(3.435e-30, RTGB_LN_315614, 1.97, RTGB_LN_2_25, 0.376, 3.72, t, eta, deta);
    else hg_fit(1.778e-29, RTGB_LN_315614, 1.965, RTGB_LN_0_541, 0.502, 2.697, t, eta, deta);
    Ls += t.T * eta * nHII;
    dLs += (eta + t.T * deta) * nHII;
    // bremsstrahlung
    double th = 1.42e-27 * t.sqrtT;
    double dth = 0.5 * th * t.invT;
    Ls += th * (nHII + nHeII + 4.0 * nHeIII);
    dLs += dth * (nHII + nHeII + 4.0 * nHeIII);
    if (helium) {
        double e2 = exp(-285335.4 * t.invT);
        double e3 = exp(-631515.0 * t.invT);
        cen_fit(9.38e-22, 285335.4, e2, t, v, dv);
        Ls += v * nHeI;
        dLs += dv * nHeI;
        // HeII: zeta + psi + eta + omega
        double zs, dzs;
        cen_fit(4.95e-22, 631515.0, e3, t, zs, dzs);
        double p2 = 5.54e-17 * t.u * exp(-0.397 * t.lnT - 473638.0 * t.invT);
        double dp2 = p2 * (-0.397 * t.invT - 0.5 * (1.0 - t.u) * t.invT + 473638.0 * t.invT * t.invT);
        double a2, da2;
        if (case_b) pow_fit(1.26e-14, RTGB_LN_570670, 0.75, t, a2, da2);
        else pow_fit(3e-14, RTGB_LN_570670, 0.654, t, a2, da2);
        double et2 = kB * t.T * a2;
        double det2 = kB * (a2 + t.T * da2);
        double e7 = exp(-94000.0 * t.invT);
        double base = 1.24e-13 * exp(-1.5 * t.lnT - 470000.0 * t.invT);
        double om = base * (1.0 + 0.3 * e7);
        double dom = om * (-1.5 * t.invT + 470000.0 * t.invT * t.invT) + base * 0.3 * e7 * 94000.0 * t.invT * t.invT;
        Ls += (zs + p2 + et2 + om) * nHeII;
        dLs += (dzs + dp2 + det2 + dom) * nHeII;
        // HeIII recombination cooling
        double e3h, de3h;
        if (case_b) hg_fit(8.0 * 3.435e-30, RTGB_LN_1263030, 1.97, RTGB_LN_2_25, 0.376, 3.72, t, e3h, de3h);
        else hg_fit(8.0 * 1.778e-29, RTGB_LN_1263030, 1.965, RTGB_LN_0_541, 0.502, 2.697, t, e3h, de3h);
        Ls += t.T * e3h * nHeIII;
        dLs += (e3h + t.T * de3h) * nHeIII;
    }
    // Compton (signed) on n_e
    double Tg = 2.727 / a_exp;
    double Tg4 = Tg * Tg * Tg * Tg;
    double vp = 1.017e-37 * Tg4 * (t.T - Tg);
    L = ne * (Ls + vp);
    dL = ne * (dLs + 1.017e-37 * Tg4);
}

}  // namespace rtgb

// Host-side checks of a state handed to rt_set_state (host pointers): gas
// fractions and temperature in range, photon densities finite and
// non-negative, |F| <= c_r N.  A large state is split over threads; the
// fault reported is the first in cell order, as a serial scan finds it.
#pragma once

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

namespace rtgb {

enum StateFault { kStateOk = 0, kStateGas = 1, kStatePhotons = 2, kStateFlux = 3 };

struct StateView {
    long long nc;
    int G;
    double cr;
    const double *nH, *xHII, *xHeII, *xHeIII, *T, *N, *F;
};

// the first faulty cell of [c0, c1): its fault, the cell in *bad
inline int check_state_range(const StateView &s, long long c0, long long c1, long long *bad)
{
    for (long long c = c0; c < c1; ++c) {
        const bool ok = std::isfinite(s.nH[c]) && s.nH[c] > 0.0 && std::isfinite(s.xHII[c]) && s.xHII[c] >= 1e-6 &&
                        s.xHII[c] <= 1.0 && s.xHeII[c] >= 0.0 && s.xHeIII[c] >= 0.0 &&
                        s.xHeII[c] + s.xHeIII[c] <= 1.0 && std::isfinite(s.T[c]) && s.T[c] > 0.0;
        if (!ok) {
            *bad = c;
            return kStateGas;
        }
        for (int g = 0; g < s.G; ++g) {
            const double n = s.N[(size_t)g * s.nc + c];
            const double fx = s.F[((size_t)3 * g) * s.nc + c], fy = s.F[((size_t)3 * g + 1) * s.nc + c],
                         fz = s.F[((size_t)3 * g + 2) * s.nc + c];
            if (!(std::isfinite(n) && n >= 0.0 && std::isfinite(fx) && std::isfinite(fy) && std::isfinite(fz))) {
                *bad = c;
                return kStatePhotons;
            }
            const double mx = std::max(std::max(std::fabs(fx), std::fabs(fy)), std::fabs(fz));
            double fm = 0.0;
            if (mx > 0.0) {
                const double a = fx / mx, b = fy / mx, d = fz / mx;
                fm = mx * std::sqrt(a * a + b * b + d * d);
            }
            if (fm > s.cr * (n * (1.0 + 1e-8) + 1e-290)) {
                *bad = c;
                return kStateFlux;
            }
        }
    }
    return kStateOk;
}

// all cells; threads for states of more than 2^16 cells
inline int check_state(const StateView &s, long long *bad)
{
    const long long kPerThread = 1LL << 15;
    long long nt = (long long)std::thread::hardware_concurrency();
    nt = std::max(1LL, std::min({nt, 16LL, s.nc / kPerThread}));
    if (nt <= 1) return check_state_range(s, 0, s.nc, bad);
    std::vector<int> kind((size_t)nt, kStateOk);
    std::vector<long long> where((size_t)nt, -1);
    std::vector<std::thread> th;
    try {
        for (long long t = 0; t < nt; ++t) {
            const long long a = s.nc * t / nt, b = s.nc * (t + 1) / nt;
            th.emplace_back([&s, &kind, &where, t, a, b] { kind[t] = check_state_range(s, a, b, &where[t]); });
        }
    } catch (...) {   // no threads to be had: the rest in this one
        const long long done = (long long)th.size();
        for (auto &x : th) x.join();
        for (long long t = 0; t < done; ++t)
            if (kind[t]) { *bad = where[t]; return kind[t]; }
        return check_state_range(s, s.nc * done / nt, s.nc, bad);
    }
    for (auto &x : th) x.join();
    for (long long t = 0; t < nt; ++t)
        if (kind[t]) {
            *bad = where[t];
            return kind[t];
        }
    return kStateOk;
}

}  // namespace rtgb

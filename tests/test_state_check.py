"""The host-side check of a state handed to rt_set_state
(paper_1304_7126_gb300/csrc/state_check.h) on the CPU: split over threads,
it must report the same fault and the same first faulty cell as a serial
scan, for valid states and for faults of every kind planted at random
cells, on sizes below, at and above the threading threshold."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1304_7126_gb300", "csrc", "state_check.h")

HARNESS = r'''
#include "state_check.h"
#include <cmath>
#include <cstdio>
#include <random>
using namespace rtgb;
int main() {
    std::mt19937_64 rng(7);
    int fails = 0, cases = 0, faults = 0;
    for (long long nc : {1LL, 100LL, 65535LL, 65536LL, 65537LL, 300001LL, 1LL << 20}) {
        for (int G : {1, 3}) {
            std::vector<double> nH(nc, 1e-3), x(nc, 0.5), y2(nc, 0.1), y3(nc, 0.1), T(nc, 1e4),
                N((size_t)G * nc, 1e-5), F((size_t)3 * G * nc, 0.0);
            const double cr = 3e9;
            for (size_t i = 0; i < F.size(); ++i) F[i] = 1e-5 * cr * 0.5 * ((i % 5) / 5.0);
            const StateView s{nc, G, cr, nH.data(), x.data(), y2.data(), y3.data(), T.data(), N.data(), F.data()};
            for (int trial = 0; trial < 10; ++trial) {
                std::vector<std::pair<std::vector<double> *, size_t>> at;
                std::vector<double> old;
                const int nf = trial == 0 ? 0 : (int)(rng() % 3) + 1;
                for (int k = 0; k < nf; ++k) {
                    const long long c = (long long)(rng() % nc);
                    std::vector<double> *a; size_t i; double v;
                    switch ((int)(rng() % 6)) {
                    case 0: a = &x; i = c; v = 2.0; break;
                    case 1: a = &T; i = c; v = -1.0; break;
                    case 2: a = &N; i = (size_t)(rng() % G) * nc + c; v = NAN; break;
                    case 3: a = &F; i = (size_t)(rng() % (3 * G)) * nc + c; v = 1.0; break;
                    case 4: a = &y2; i = c; v = 0.95; break;
                    default: a = &nH; i = c; v = 0.0; break;
                    }
                    at.push_back({a, i}); old.push_back((*a)[i]); (*a)[i] = v;
                }
                long long b1 = -1, b2 = -1;
                const int k1 = check_state_range(s, 0, nc, &b1), k2 = check_state(s, &b2);
                ++cases; faults += k1 != 0;
                if (k1 != k2 || (k1 && b1 != b2)) ++fails;
                for (int k = nf - 1; k >= 0; --k) (*at[k].first)[at[k].second] = old[k];
            }
        }
    }
    printf("%d %d %d\n", cases, faults, fails);
    return 0;
}
'''


def test_threaded_state_check_matches_serial(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    src = tmp_path / "harness.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "harness"
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-pthread", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    cases, faults, fails = map(int, out)
    assert cases == 140 and faults > 100 and fails == 0, out

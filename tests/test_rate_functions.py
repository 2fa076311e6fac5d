"""The thermochemistry kernels' rate functions against the oracle's rate
fits (CPU).

On the GPU every rate coefficient and cooling term of App. A is one
function f(T) = Cc exp(c0 + c1 ln T + c2/T - c3 ln(1 + exp(c4 ln T + c5))),
its constants derived at compile time from the fit constants (Cen's
A sqrt(T) u e^(-T0/T) with ln u = -ln(1 + sqrt(T/1e5)), the Hui & Gnedin
forms A lam^p / (1 + (lam/l0)^r)^s, the power law of alpha_HeII, and the
products that make the cooling terms).  rt_rate_functions returns those
constants as the kernels hold them; evaluated here in float64, each
function must equal the oracle's fit (written independently, in the
printed form) to 1e-12 and its T-derivative, d ln f/dT = (c1 - c2/T -
c3 c4 sigma)/T, the oracle's to 1e-10, from 10 K to 1e8 K, for both
recombination cases.  The remaining slots are zero."""
import numpy as np
import pytest

# slot -> oracle rate names summed into it (the two omega_HeII terms are
# separate slots)
SLOTS = {
    0: ["zeta_HI"], 1: ["psi_HI"], 2: ["eta_HII"], 3: ["theta"], 4: ["zeta_HeI"], 5: ["zeta_HeII"],
    6: ["psi_HeII"], 7: ["eta_HeII"], 10: ["eta_HeIII"],
    16: ["beta_HI"], 17: ["alpha_HII"], 18: ["beta_HeI"], 19: ["beta_HeII"], 20: ["alpha_HeII"],
    21: ["alpha_HeIII"],
}
OMEGA = (8, 9)


def _eval(c, T):
    Cc, c0, c1, c2, c3, c4, c5 = c
    lnT = np.log(T)
    z = c4 * lnT + c5
    sp = np.logaddexp(0.0, z)
    sig = 0.5 * (1.0 + np.tanh(0.5 * z))
    f = Cc * np.exp(c0 + c1 * lnT + c2 / T - c3 * sp)
    df = f * (c1 - c2 / T - c3 * c4 * sig) / T
    return f, df


@pytest.fixture(scope="module")
def R():
    from paper_1304_7126_gb300 import rt
    rt.load()
    return rt


@pytest.mark.parametrize("case_b", [True, False])
def test_rate_functions_equal_the_oracle_fits(R, oracle_mod, case_b):
    tab = R.rate_functions(case_b)
    Ts = np.geomspace(10.0, 1e8, 61)
    worst, worst_d = 0.0, 0.0
    for T in Ts:
        r, dr = oracle_mod.rates(T, 1.0, case_b)
        vals = {k: _eval(tab[k], T) for k in range(32)}
        pairs = [(vals[k], sum(r[n] for n in names), sum(dr[n] for n in names)) for k, names in SLOTS.items()]
        f8, d8 = vals[OMEGA[0]]
        f9, d9 = vals[OMEGA[1]]
        pairs.append(((f8 + f9, d8 + d9), r["omega_HeII"], dr["omega_HeII"]))
        for (f, df), ref, dref in pairs:
            if ref > 1e-280:
                worst = max(worst, abs(f - ref) / ref)
            if abs(dref) > 1e-280 and ref > 1e-280:
                worst_d = max(worst_d, abs(df - dref) / abs(dref))
    assert worst < 1e-12, worst
    assert worst_d < 1e-10, worst_d
    for k in list(range(11, 16)) + list(range(22, 32)):
        assert tab[k][0] == 0.0, k


def test_rate_functions_rejects_bad_arguments(R):
    import ctypes as C
    L = R.load()
    out = np.zeros((32, 7))
    assert L.rt_rate_functions(2, out.ctypes.data_as(C.c_void_p)) == R.RT_EINVAL
    assert L.rt_rate_functions(1, None) == R.RT_EINVAL

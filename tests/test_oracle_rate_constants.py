"""The oracle's rate fits against the paper's printed constants, taken
mechanically from the paper's LaTeX source (tests/golden/rate_constants.json,
written by tests/golden/extract_rate_constants.py; no constant below is
typed by hand), evaluated here in 50-digit arithmetic.  A constant mistyped
in the oracle fails this test.

The shape of each fit is the one printed in the appendix on interaction
rate coefficients: Cen (1992) forms A sqrt(T) (1 + sqrt(T/1e5))^-1
exp(-T0/T) (collisional ionisation beta, its cooling zeta) and A T^p
(1 + sqrt(T/1e5))^-1 exp(-T0/T) (collisional excitation psi); Hui & Gnedin
(1997) forms A lam^p / (1 + (lam/l0)^r)^s (recombination alpha; times T for
the recombination cooling eta), lam = T_lam/T with the lambda of the
subscript printed in the fit; power laws A lam^p (alpha_HeII); eta_HeII =
k_B T alpha_HeII; theta = A sqrt(T) (the factor 4 of HeIII is a weight in
the cooling sum); Compton A (T_g/a)^4 (T - T_g/a); dielectronic A T^p
exp(-T1/T) (1 + B exp(-T2/T))."""
import json
import os
import re

import pytest

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rate_constants.json")))["fits"]
K_B = "1.380649e-16"
TGRID = [30.0, 300.0, 3e3, 1e4, 3e4, 1e5, 1e6, 1e7]


def _fit(name):
    return GOLD[name]


def _lam_of(mp, fit):
    """lam(T) of the subscript printed on lambda in this fit."""
    sub = re.search(r"\\lambda\^\{[-\d.]+\}_\{\\(\w+)\}", fit["latex"]).group(1)
    t = mp.mpf(_fit(r"\lambda_{\%s}(T)" % sub)["numbers"][0])
    return lambda T: t / T


def _model(mp):
    """name in the oracle -> (case A fit, case B fit) as functions of T."""
    V = lambda f, i: mp.mpf(f["numbers"][i])  # noqa: E731

    def cen(f, with_sqrt):
        A, one, T5, m1, T0 = (V(f, i) for i in range(5))
        assert one == 1 and m1 == -1
        return lambda T: A * (mp.sqrt(T) if with_sqrt else 1) * (1 + mp.sqrt(T / T5)) ** m1 * mp.exp(T0 / T)

    def psi_he(f):
        A, p, one, T5, m1, T0 = (V(f, i) for i in range(6))
        return lambda T: A * T ** p * (one + mp.sqrt(T / T5)) ** m1 * mp.exp(T0 / T)

    def hg(f, times_T, lead=1):
        off = 1 if lead != 1 else 0
        pre = V(f, 0) if off else 1
        A, p, one, l0, r, s = (V(f, off + i) for i in range(6))
        lam = _lam_of(mp, f)
        return lambda T: pre * A * (T if times_T else 1) * lam(T) ** p / (one + (lam(T) / l0) ** r) ** s

    def pw(f, times_kT=False):
        A, p = V(f, 0), V(f, 1)
        lam = _lam_of(mp, f)
        kb = mp.mpf(K_B)
        return lambda T: (kb * T if times_kT else 1) * A * lam(T) ** p

    m = {}
    for sp, key in (("HI", "hi"), ("HeI", "hei"), ("HeII", "heii")):
        m["beta_" + sp] = (cen(_fit(r"\beta_{\%s}(T)" % key), True),) * 2
        m["zeta_" + sp] = (cen(_fit(r"\zeta_{\%s}(T)" % key), True),) * 2
    m["alpha_HII"] = (hg(_fit(r"\recA_{\hii}(T)"), False), hg(_fit(r"\recB_{\hii}(T)"), False))
    m["alpha_HeII"] = (pw(_fit(r"\recA_{\heii}(T)")), pw(_fit(r"\recB_{\heii}(T)")))
    m["alpha_HeIII"] = (hg(_fit(r"\recA_{\heiii}(T)"), False), hg(_fit(r"\recB_{\heiii}(T)"), False))
    m["eta_HII"] = (hg(_fit(r"\eta^{A}_{\hii}(T)"), True), hg(_fit(r"\eta^{B}_{\hii}(T)"), True))
    m["eta_HeII"] = (pw(_fit(r"\eta^{A}_{\heii}(T)"), True), pw(_fit(r"\eta^{B}_{\heii}(T)"), True))
    m["eta_HeIII"] = (hg(_fit(r"\eta^{A}_{\heiii}(T)"), True, lead=8), hg(_fit(r"\eta^{B}_{\heiii}(T)"), True, lead=8))
    m["psi_HI"] = (cen(_fit(r"\psi_{\hi}(T)"), False),) * 2
    m["psi_HeII"] = (psi_he(_fit(r"\psi_{\heii}(T)")),) * 2
    th = _fit(r"\theta_{\hii}(T)")
    assert _fit(r"\theta_{\heii}(T)")["numbers"] == th["numbers"]
    assert _fit(r"\theta_{\heiii}(T)")["numbers"] == ["4"] + th["numbers"]
    m["theta"] = (lambda T: V(th, 0) * mp.sqrt(T),) * 2
    om = _fit(r"\omega_{\heii}(T)")
    A, p, T1, one, B, T2 = (V(om, i) for i in range(6))
    m["omega_HeII"] = (lambda T: A * T ** p * mp.exp(T1 / T) * (one + B * mp.exp(T2 / T)),) * 2
    return m


def test_extracted_layout():
    """The extraction found every fit with the number of constants its form has."""
    n = {k: len(v["numbers"]) for k, v in GOLD.items()}
    assert n[r"\beta_{\hi}(T)"] == 5 and n[r"\recB_{\hii}(T)"] == 6 and n[r"\eta^{B}_{\heiii}(T)"] == 7
    assert n[r"\omega_{\heii}(T)"] == 6 and n[r"\varpi(T,a)"] == 4 and len(GOLD) == 28


@pytest.mark.parametrize("case_b", [False, True])
def test_fits_equal_printed_constants(oracle_mod, case_b):
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 50
    model = _model(mp)
    for T in TGRID:
        r, _ = oracle_mod.rates(T, case_b=case_b)
        for name, fns in model.items():
            want = fns[1 if case_b else 0](mp.mpf(T))
            got = r[name]
            if want == 0:
                assert got == 0.0, (name, T)
                continue
            if abs(want) < mp.mpf("1e-300"):   # below the double range: the oracle underflows
                assert abs(got) < 1e-290, (name, T)
                continue
            assert abs(mp.mpf(got) / want - 1) < 1e-13, (name, T, got, float(want))


def test_compton_printed_constants(oracle_mod):
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 50
    f = _fit(r"\varpi(T,a)")
    A, Tg, four, Tg2 = (mp.mpf(v) for v in f["numbers"])
    assert Tg == Tg2 and four == 4
    for a in (1.0, 0.25):
        for T in (10.0, 1e4, 1e6):
            want = A * (Tg / a) ** four * (T - Tg / a)
            got = oracle_mod.rates(T, a_exp=a)[0]["varpi"]
            assert abs(mp.mpf(got) / want - 1) < 1e-13, (a, T)

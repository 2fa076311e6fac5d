"""The double-float exp/log tables and split constants (dfmath_tables.h) are
what their definitions give: regenerating them with gen_dfmath_tables.py
(60-digit mpmath values of 2^(j/64), ln(1 + j/128), 1/(1 + j/128) and the
ln 2 splits, each split into a pair of floats) reproduces the committed
header byte for byte; and each pair sums to its value within 2^-48."""
import os
import subprocess
import sys

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1304_7126_gb300", "csrc")


def test_tables_regenerate():
    pytest.importorskip("mpmath")
    out = subprocess.run([sys.executable, "gen_dfmath_tables.py"], cwd=CSRC, capture_output=True, text=True,
                         check=True).stdout
    with open(os.path.join(CSRC, "dfmath_tables.h")) as f:
        assert out.strip() == f.read().strip()


def test_pairs_sum_to_their_values():
    mpmath = pytest.importorskip("mpmath")
    import re
    mpmath.mp.dps = 40
    with open(os.path.join(CSRC, "dfmath_tables.h")) as f:
        text = f.read()
    num = r"(-?0x[0-9a-fp.+-]+f|0\.0f)"
    h = lambda s: float.fromhex(s[:-1]) if s != "0.0f" else 0.0  # noqa: E731
    exp_rows = re.findall(r"\{%s, %s\}" % (num, num), text.split("kDfExp2Tab")[1].split("};")[0])
    assert len(exp_rows) == 64
    for j, (hi, lo) in enumerate(exp_rows):
        v = mpmath.mpf(h(hi)) + mpmath.mpf(h(lo))
        assert abs(v / mpmath.power(2, mpmath.mpf(j) / 64) - 1) < mpmath.mpf(2) ** -48
    log_rows = re.findall(r"\{%s, %s, %s, %s\}" % (num, num, num, num), text.split("kDfLogTab")[1].split("};")[0])
    assert len(log_rows) == 129
    for j, row in enumerate(log_rows):
        F = 1 + mpmath.mpf(j) / 128
        lnF = mpmath.mpf(h(row[0])) + mpmath.mpf(h(row[1]))
        inv = mpmath.mpf(h(row[2])) + mpmath.mpf(h(row[3]))
        assert abs(lnF - mpmath.log(F)) <= mpmath.mpf(2) ** -48 * max(mpmath.log(F), mpmath.mpf(2) ** -8)
        assert abs(inv * F - 1) < mpmath.mpf(2) ** -47


def test_softplus_polynomials():
    """The softplus table's pair coefficients give ln(1 + e^z) within
    2e-14 absolute (the pair precision of the constant term at |z| ~ 16)
    and its derivative 1/(1 + e^-z) within 1e-14, at 13 points of every
    fourth interval of [-16, 16)."""
    mpmath = pytest.importorskip("mpmath")
    import re
    mpmath.mp.dps = 40
    with open(os.path.join(CSRC, "dfmath_tables.h")) as f:
        text = f.read()
    num = r"(-?0x[0-9a-fp.+-]+f|0\.0f)"
    h = lambda s: float.fromhex(s[:-1]) if s != "0.0f" else 0.0  # noqa: E731
    lo, per, n, deg = (int(v) for v in re.search(
        r"kDfSpLo = (-?\d+), kDfSpPer = (\d+), kDfSpN = (\d+), kDfSpDeg = (\d+)", text).groups())
    body = text.split("kDfSoftplusTab")[1].split("};")[0]
    pairs = re.findall(r"\{%s, %s\}" % (num, num), body)
    assert len(pairs) == n * (deg + 1)
    for k in range(0, n, 4):
        c = [mpmath.mpf(h(a)) + mpmath.mpf(h(b)) for a, b in pairs[k * (deg + 1):(k + 1) * (deg + 1)]]
        mid = lo + (mpmath.mpf(k) + mpmath.mpf(1) / 2) / per
        for i in range(13):
            t = (mpmath.mpf(i) / 12 - mpmath.mpf(1) / 2) / per
            z = mid + t
            P = sum(c[j] * t ** j for j in range(deg + 1))
            D = sum(j * c[j] * t ** (j - 1) for j in range(1, deg + 1))
            assert abs(P - mpmath.log1p(mpmath.exp(z))) < 2e-14
            assert abs(D - 1 / (1 + mpmath.exp(-z))) < 1e-14

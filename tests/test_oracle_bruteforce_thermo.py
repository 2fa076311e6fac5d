"""One accepted thermochemistry sub-step of a hydrogen cell (X = 1, two
photon groups, evolving T, case B / OTSA) in the oracle against a
brute-force evaluation in 50-digit arithmetic (mpmath), written here from
the paper's App. A in its order and the fits of its rate appendix:
  1. N' = N / (1 + h D), F' = F / (1 + h D), D = c_r sigma^N n_HI;
  2. T/mu' = T/mu + Lambda K h / (1 - Lambda' K h), Lambda = heating with N'
     (Eq. (PHeat2)) minus the cooling of Eq. (rate_cooling) at T(t),
     Lambda' = mu dLambda/dT, K = (gamma - 1) X / (n_H k_B);
  3. x' = x + h (C - x (C + D)) / (1 - J h) with the rates at
     T' = (T/mu)' mu(x(t)) and J from dC/dx, dD/dx including the
     temperature terms;
  4. T = (T/mu)' mu(x').
The rates' temperature derivatives are taken numerically at 50 digits, not
from the oracle's analytic forms.  Oracle and brute force agree to 1e-12."""
import numpy as np
import pytest

C = 2.99792458e10
EV = 1.602176634e-12
K_B = 1.380649e-16


def _rates(mp):
    lam = lambda T: mp.mpf(315614) / T  # noqa: E731
    cen = lambda T: 1 / (1 + mp.sqrt(T / mp.mpf(10) ** 5))  # noqa: E731
    return {
        "alpha": lambda T: mp.mpf("2.753e-14") * lam(T) ** mp.mpf("1.5") /
        (1 + (lam(T) / mp.mpf("2.74")) ** mp.mpf("0.407")) ** mp.mpf("2.242"),
        "beta": lambda T: mp.mpf("5.85e-11") * mp.sqrt(T) * cen(T) * mp.exp(-mp.mpf("157809.1") / T),
        "zeta": lambda T: mp.mpf("1.27e-21") * mp.sqrt(T) * cen(T) * mp.exp(-mp.mpf("157809.1") / T),
        "psi": lambda T: mp.mpf("7.5e-19") * cen(T) * mp.exp(-mp.mpf(118348) / T),
        "eta": lambda T: mp.mpf("3.435e-30") * T * lam(T) ** mp.mpf("1.97") /
        (1 + (lam(T) / mp.mpf("2.25")) ** mp.mpf("0.376")) ** mp.mpf("3.72"),
        "theta": lambda T: mp.mpf("1.42e-27") * mp.sqrt(T),
        "compton": lambda T: mp.mpf("1.017e-37") * mp.mpf("2.727") ** 4 * (T - mp.mpf("2.727")),
    }


def _substep(mp, nH, x, T, N, F, h, cr, sigN, sigE, egy):
    r = _rates(mp)
    nH, x, T, h, cr = (mp.mpf(v) for v in (nH, x, T, h, cr))
    G = len(N)
    nHI, ne = nH * (1 - x), nH * x
    # 1. photons
    inv = [1 / (1 + h * cr * mp.mpf(sigN[i]) * nHI) for i in range(G)]
    N1 = [mp.mpf(N[i]) * inv[i] for i in range(G)]
    F1 = [[mp.mpf(F[i][d]) * inv[i] for d in range(3)] for i in range(G)]
    # 2. temperature
    e0 = mp.mpf("13.60") * mp.mpf(EV)
    heat = sum(nHI * cr * N1[i] * (mp.mpf(egy[i]) * mp.mpf(sigE[i]) - e0 * mp.mpf(sigN[i])) for i in range(G))
    cool = lambda TT: ne * ((r["zeta"](TT) + r["psi"](TT)) * nHI + (r["eta"](TT) + r["theta"](TT)) * nH * x  # noqa: E731
                            + r["compton"](TT))
    mu = 1 / (1 + x)
    K = (mp.mpf(5) / 3 - 1) / (nH * mp.mpf(K_B))
    lam_ = heat - cool(T)
    dlam = -mu * mp.diff(cool, T)
    Tmu1 = T / mu + lam_ * K * h / (1 - dlam * K * h)
    # 3. hydrogen, rates at T' = (T/mu)' mu(x(t))
    T1 = Tmu1 * mu
    al, be = r["alpha"](T1), r["beta"](T1)
    dal, dbe = mp.diff(r["alpha"], T1), mp.diff(r["beta"], T1)
    Cc = be * ne + sum(mp.mpf(sigN[i]) * cr * N1[i] for i in range(G))
    Dd = al * ne
    dC = nH * be - ne * Tmu1 * mu * mu * dbe
    dD = nH * al - ne * Tmu1 * mu * mu * dal
    J = dC - (Cc + Dd) - x * (dC + dD)
    x1 = x + h * (Cc - x * (Cc + Dd)) / (1 - J * h)
    x1 = min(max(x1, mp.mpf("1e-6")), mp.mpf(1))
    T2 = max(Tmu1 / (1 + x1), mp.mpf(1))
    return x1, T2, N1, F1


@pytest.mark.parametrize("x0,T0,h", [(1e-3, 3e3, 3e7), (0.3, 1.5e4, 1e8), (0.95, 8e4, 1e9)])
def test_thermo_substep_vs_50_digits(oracle_mod, x0, T0, h):
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 50
    O = oracle_mod
    cr = C / 10.0
    sigN = (3.0e-18, 5.7e-19)
    sigE = (2.8e-18, 5.0e-19)
    egy = (18.85 * EV, 35.08 * EV)
    p = O.Problem((1, 1, 1), 1e20, 2, cr, [[s, 0, 0] for s in sigN], [[s, 0, 0] for s in sigE], egy, X=1.0,
                  isothermal=False, otsa=True)
    nH = 0.05
    N = [2e-6, 5e-7]
    F = [[cr * N[0] * 0.3, -cr * N[0] * 0.2, cr * N[0] * 0.1], [0.0, cr * N[1] * 0.5, 0.0]]
    st, s, N1, F1, att, _, _ = p.thermo_cell(h, nH, [x0, 0.0, 0.0, T0], N, np.array(F))
    assert st == 0 and att == 1     # a single accepted sub-step
    x1, T1, Nm, Fm = _substep(mp, nH, x0, T0, N, F, h, cr, sigN, sigE, egy)
    assert abs(s[0] / float(x1) - 1) < 1e-12
    assert abs(s[3] / float(T1) - 1) < 1e-12
    for i in range(2):
        assert abs(N1[i] / float(Nm[i]) - 1) < 1e-13
        for d in range(3):
            assert abs(F1[i][d] - float(Fm[i][d])) <= 1e-13 * cr * float(Nm[i])
    assert s[1] == 0.0 and s[2] == 0.0

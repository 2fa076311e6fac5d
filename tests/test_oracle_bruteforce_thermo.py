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


def _rates_he(mp):
    cen = lambda T: 1 / (1 + mp.sqrt(T / mp.mpf(10) ** 5))  # noqa: E731
    l1 = lambda T: mp.mpf(570670) / T  # noqa: E731
    l2 = lambda T: mp.mpf(1263030) / T  # noqa: E731
    return {
        "aHeII": lambda T: mp.mpf("1.26e-14") * l1(T) ** mp.mpf("0.75"),
        "aHeIII": lambda T: mp.mpf("5.506e-14") * l2(T) ** mp.mpf("1.5") /
        (1 + (l2(T) / mp.mpf("2.74")) ** mp.mpf("0.407")) ** mp.mpf("2.242"),
        "bHeI": lambda T: mp.mpf("2.38e-11") * mp.sqrt(T) * cen(T) * mp.exp(-mp.mpf("285335.4") / T),
        "bHeII": lambda T: mp.mpf("5.68e-12") * mp.sqrt(T) * cen(T) * mp.exp(-mp.mpf(631515) / T),
        "zHeI": lambda T: mp.mpf("9.38e-22") * mp.sqrt(T) * cen(T) * mp.exp(-mp.mpf("285335.4") / T),
        "zHeII": lambda T: mp.mpf("4.95e-22") * mp.sqrt(T) * cen(T) * mp.exp(-mp.mpf(631515) / T),
        "pHeII": lambda T: mp.mpf("5.54e-17") * T ** mp.mpf("-0.397") * cen(T) * mp.exp(-mp.mpf(473638) / T),
        "eHeII": lambda T: mp.mpf(K_B) * T * mp.mpf("1.26e-14") * l1(T) ** mp.mpf("0.75"),
        "oHeII": lambda T: mp.mpf("1.24e-13") * T ** mp.mpf("-1.5") * mp.exp(-mp.mpf(470000) / T) *
        (1 + mp.mpf("0.3") * mp.exp(-mp.mpf(94000) / T)),
        "eHeIII": lambda T: 8 * mp.mpf("3.435e-30") * T * l2(T) ** mp.mpf("1.97") /
        (1 + (l2(T) / mp.mpf("2.25")) ** mp.mpf("0.376")) ** mp.mpf("3.72"),
    }


def _substep_he(mp, X, nH, x, y2, y3, T, N, h, cr, sigN, sigE, egy):
    """sigN, sigE [G][3] (HI, HeI, HeII); returns x, y2, y3, T, N'."""
    r, q = _rates(mp), _rates_he(mp)
    X, nH, x, y2, y3, T, h, cr = (mp.mpf(v) for v in (X, nH, x, y2, y3, T, h, cr))
    G = len(N)
    nHe = nH * (1 - X) / (4 * X)
    mden = lambda a, b, c: X * (1 + a) + (1 - X) / 4 * (1 + b + 2 * c)  # noqa: E731  1/mu
    n = [nH * (1 - x), nHe * (1 - y2 - y3), nHe * y2]          # HI, HeI, HeII absorbers
    ne = x * nH + (y2 + 2 * y3) * nHe
    sN = [[mp.mpf(v) for v in row] for row in sigN]
    sE = [[mp.mpf(v) for v in row] for row in sigE]
    N1 = [mp.mpf(N[i]) / (1 + h * cr * sum(sN[i][j] * n[j] for j in range(3))) for i in range(G)]
    eps = [mp.mpf(v) * mp.mpf(EV) for v in ("13.60", "24.59", "54.42")]
    heat = sum(n[j] * cr * N1[i] * (mp.mpf(egy[i]) * sE[i][j] - eps[j] * sN[i][j]) for i in range(G) for j in range(3))
    nHII, nHeIII = nH * x, nHe * y3

    def cool(TT):
        return ne * ((r["zeta"](TT) + r["psi"](TT)) * n[0] + q["zHeI"](TT) * n[1]
                     + (q["zHeII"](TT) + q["pHeII"](TT) + q["eHeII"](TT) + q["oHeII"](TT)) * n[2]
                     + r["eta"](TT) * nHII + q["eHeIII"](TT) * nHeIII
                     + r["theta"](TT) * (nHII + n[2] + 4 * nHeIII) + r["compton"](TT))

    mu = 1 / mden(x, y2, y3)
    K = (mp.mpf(5) / 3 - 1) * X / (nH * mp.mpf(K_B))
    lam_ = heat - cool(T)
    dlam = -mu * mp.diff(cool, T)
    Tmu1 = T / mu + lam_ * K * h / (1 - dlam * K * h)
    # hydrogen at T' = (T/mu)' mu(x(t))
    T1 = Tmu1 * mu
    al, be = r["alpha"](T1), r["beta"](T1)
    dal, dbe = mp.diff(r["alpha"], T1), mp.diff(r["beta"], T1)
    g = [sum(sN[i][j] * cr * N1[i] for i in range(G)) for j in range(3)]   # photoionisation rates
    Cc = be * ne + g[0]
    Dd = al * ne
    dC = nH * be - ne * Tmu1 * mu * mu * X * dbe
    dD = nH * al - ne * Tmu1 * mu * mu * X * dal
    J = dC - (Cc + Dd) - x * (dC + dD)
    x1 = min(max(x + h * (Cc - x * (Cc + Dd)) / (1 - J * h), mp.mpf("1e-6")), mp.mpf(1))
    # helium, n_e and T refreshed with the forward values before each update
    yI = 1 - y2 - y3
    ne2 = x1 * nH + (y2 + 2 * y3) * nHe
    T2 = Tmu1 / mden(x1, y2, y3)
    yI1 = (yI + y2 * q["aHeII"](T2) * ne2 * h) / (1 + (q["bHeI"](T2) * ne2 + g[1]) * h)
    C2 = yI1 * (q["bHeI"](T2) * ne2 + g[1]) + y3 * q["aHeIII"](T2) * ne2
    D2 = (q["bHeII"](T2) + q["aHeII"](T2)) * ne2 + g[2]
    y2n = (y2 + C2 * h) / (1 + D2 * h)
    ne3 = x1 * nH + (y2n + 2 * y3) * nHe
    T3 = Tmu1 / mden(x1, y2n, y3)
    y3n = (y3 + y2n * (q["bHeII"](T3) * ne3 + g[2]) * h) / (1 + q["aHeIII"](T3) * ne3 * h)
    # conservation: the largest fraction takes 1 minus the other two
    if y2n >= yI1 and y2n >= y3n:
        y2n = 1 - yI1 - y3n
    elif y3n >= yI1 and y3n > y2n:
        y3n = 1 - yI1 - y2n
    y2n = min(max(y2n, mp.mpf(0)), mp.mpf(1))
    y3n = min(max(y3n, mp.mpf(0)), mp.mpf(1))
    Tf = max(Tmu1 / mden(x1, y2n, y3n), mp.mpf(1))
    return x1, y2n, y3n, Tf, N1


@pytest.mark.parametrize("x0,y20,y30,T0,h,N", [
    (1e-3, 1e-3, 1e-6, 3e3, 3e7, (2e-6, 5e-7, 1e-7)),
    (0.5, 0.4, 0.05, 2e4, 1e8, (2e-6, 5e-7, 1e-7)),
    (0.99, 0.2, 0.75, 6e4, 3e8, (2e-6, 5e-7, 1e-7)),      # HeIII largest: renormalised
    (0.99, 0.9, 0.05, 3e4, 4e9, (1e-8, 1e-8, 8e-4)),      # HeII -> HeIII by ~1% within the sub-step
])
def test_thermo_substep_helium_vs_50_digits(oracle_mod, x0, y20, y30, T0, h, N):
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 50
    O = oracle_mod
    cr = C / 10.0
    # three bands as in the cosmological workload (HeI and HeII absorb only above their thresholds)
    sigN = [[3.0e-18, 0.0, 0.0], [5.7e-19, 4.5e-18, 0.0], [7.9e-20, 1.2e-18, 1.06e-18]]
    sigE = [[2.8e-18, 0.0, 0.0], [5.0e-19, 4.1e-18, 0.0], [7.5e-20, 1.1e-18, 1.0e-18]]
    egy = (18.85 * EV, 35.08 * EV, 65.66 * EV)
    X = 0.76
    p = O.Problem((1, 1, 1), 1e20, 3, cr, sigN, sigE, egy, X=X, isothermal=False, otsa=True)
    nH = 0.05
    N = list(N)
    st, s, N1, _, att, _, _ = p.thermo_cell(h, nH, [x0, y20, y30, T0], N, np.zeros((3, 3)))
    assert st == 0 and att == 1
    x1, y2, y3, T1, Nm = _substep_he(mp, X, nH, x0, y20, y30, T0, N, h, cr, sigN, sigE, egy)
    for got, ref in ((s[0], x1), (s[1], y2), (s[2], y3), (s[3], T1)):
        assert abs(got - float(ref)) <= 1e-12 * max(abs(float(ref)), 1e-6), (got, float(ref))
    for i in range(3):
        assert abs(N1[i] / float(Nm[i]) - 1) < 1e-13

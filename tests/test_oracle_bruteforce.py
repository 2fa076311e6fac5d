"""One transport step of the oracle on a 4^3 periodic box against a
brute-force evaluation of the same step in 50-digit arithmetic (mpmath),
written here from the paper's equations: the M1 closure (Sec. 2, Eqs.
(edd2), (eddTens), (Udir)), the GLF (Eq. (glf)) or HLL (Eq. (hll)) face
flux, with the HLL speeds interpolated bilinearly in the same table, and the
unsplit update of Eq. (dUdt_sol).  It checks the oracle's C implementation
(indexing, ghost cells, signs, the order of the sums) to 1e-13, beyond what
the conservation and symmetry pins see."""
import numpy as np
import pytest

C = 2.99792458e10


def _closure(mp, c, N, F):
    """f, n and the pressure tensor c^2 N D of one cell."""
    Fm = mp.sqrt(F[0] ** 2 + F[1] ** 2 + F[2] ** 2)
    if N > mp.mpf("1e-30") and Fm > 0:
        f = min(Fm / (c * N), mp.mpf(1))
        n = [F[i] / Fm for i in range(3)]
    else:
        f = mp.mpf(0)
        n = [mp.mpf(0)] * 3
    chi = (3 + 4 * f * f) / (5 + 2 * mp.sqrt(4 - 3 * f * f))
    a = (1 - chi) / 2
    b = (3 * chi - 1) / 2
    P = [[c * c * N * ((a if i == j else 0) + b * n[i] * n[j]) for j in range(3)] for i in range(3)]
    return f, n, P


def _speeds(mp, tab, f, mu):
    nf, nmu = tab.shape[0], tab.shape[1]
    fx = f * (nf - 1)
    k = min(max(int(mp.floor(fx)), 0), nf - 2)
    wf = fx - k
    mx = (mu + 1) / 2 * (nmu - 1)
    j = min(max(int(mp.floor(mx)), 0), nmu - 2)
    wm = mx - j
    out = []
    for q in range(2):
        a, b = mp.mpf(tab[k, j, q]), mp.mpf(tab[k, j + 1, q])
        c_, d = mp.mpf(tab[k + 1, j, q]), mp.mpf(tab[k + 1, j + 1, q])
        v0 = a + wm * (b - a)
        v1 = c_ + wm * (d - c_)
        out.append(v0 + wf * (v1 - v0))
    return out[0], out[1]


def _step_mp(mp, shape, G, c, dt, dx, N, F, flux, tab):
    nz, ny, nx = shape
    nc = nz * ny * nx
    Nn = np.empty(G * nc, dtype=object)
    Fn = np.empty(3 * G * nc, dtype=object)
    idx = lambda z, y, x: (z % nz) * ny * nx + (y % ny) * nx + (x % nx)  # noqa: E731
    for g in range(G):
        U, Q = {}, {}
        for cidx in range(nc):
            u = [mp.mpf(N[g * nc + cidx])] + [mp.mpf(F[(3 * g + i) * nc + cidx]) for i in range(3)]
            U[cidx] = u
            Q[cidx] = _closure(mp, c, u[0], u[1:])

        def phi(cidx, d):
            u = U[cidx]
            P = Q[cidx][2]
            return [u[1 + d]] + [P[i][d] for i in range(3)]

        def face(L, R, d):
            fL, fR = phi(L, d), phi(R, d)
            uL, uR = U[L], U[R]
            if flux == 0:
                return [(fL[q] + fR[q]) / 2 - c / 2 * (uR[q] - uL[q]) for q in range(4)]
            loL, hiL = _speeds(mp, tab, Q[L][0], Q[L][1][d])
            loR, hiR = _speeds(mp, tab, Q[R][0], Q[R][1][d])
            lp = max(mp.mpf(0), c * hiL, c * hiR)
            lm = min(mp.mpf(0), c * loL, c * loR)
            return [(lp * fL[q] - lm * fR[q] + lp * lm * (uR[q] - uL[q])) / (lp - lm) for q in range(4)]

        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    cidx = idx(z, y, x)
                    acc = [mp.mpf(0)] * 4
                    for d, (oz, oy, ox) in enumerate(((0, 0, 1), (0, 1, 0), (1, 0, 0))):
                        lo = face(idx(z - oz, y - oy, x - ox), cidx, d)
                        hi = face(cidx, idx(z + oz, y + oy, x + ox), d)
                        for q in range(4):
                            acc[q] += lo[q] - hi[q]
                    u = [U[cidx][q] + dt / dx * acc[q] for q in range(4)]
                    Nn[g * nc + cidx] = u[0]
                    for i in range(3):
                        Fn[(3 * g + i) * nc + cidx] = u[1 + i]
    return Nn, Fn


@pytest.mark.parametrize("flux", [0, 1])
def test_transport_step_vs_50_digits(oracle_mod, flux):
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp
    mp.dps = 50
    O = oracle_mod
    from oracle import hll_table
    tab = hll_table.table()
    shape, G, dx = (4, 4, 4), 2, 1e20
    cr = C / 100.0
    p = O.Problem(shape, dx, G, cr, np.zeros((G, 3)), np.zeros((G, 3)), np.full(G, 3e-11), X=1.0,
                  isothermal=True, otsa=True, flux=flux, bc=(2,) * 6, skip_thermo=True, hll_table=tab)
    rng = np.random.default_rng(11 + flux)
    nc = 64
    N = 10 ** rng.uniform(-3, 0, size=(G, nc))
    d = rng.standard_normal((G, 3, nc))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    F = cr * N[:, None, :] * rng.uniform(0.0, 0.9, size=(G, 1, nc)) * d
    # every cell far above the closure floor (1e-30 photons/cm^3): the floor
    # reading leaves such a state alone, so this is also the step without it
    assert N.min() > 1e-20
    s = O.new_state(shape, G, 1e-3, 1e-6, 1e4)
    s["N"], s["F"] = N.reshape(-1).copy(), F.reshape(-1).copy()
    dt = O.courant_dt(0.8, dx, cr)
    Nm, Fm = _step_mp(mp, shape, G, mp.mpf(cr), mp.mpf(dt), mp.mpf(dx), s["N"], s["F"], flux, tab)
    st, _, _, _ = p.step(s, dt)
    assert st == 0
    Nref = np.array([float(v) for v in Nm])
    Fref = np.array([float(v) for v in Fm])
    assert np.all(np.linalg.norm(Fref.reshape(G, 3, nc), axis=1) <= cr * Nref.reshape(G, nc))   # no clamp met
    assert np.max(np.abs(s["N"] - Nref) / np.abs(Nref)) < 1e-13
    scale = np.repeat(cr * Nref.reshape(G, 1, nc), 3, axis=1).reshape(-1)
    assert np.max(np.abs(s["F"] - Fref) / scale) < 1e-13

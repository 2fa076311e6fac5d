"""Closed-form references and diagnostics used by the tests.

Stromgren sphere (Sec. 4.2, Eq. (Stromgren_radius); Sec. 6 test 1,
Eq. (r_analyt)), the relativistic front law of Shapiro et al. quoted in
Sec. 4.2 (Eq. (Stromgr_w_rel)), photo-ionisation and collisional equilibria
of the hydrogen rate equation (Sec. 3.3, Eq. (thchem_xhii) with
dx/dt = 0), and the I-front radius diagnostic used in Sec. 6 (radius where
the spherically averaged ionised fraction crosses 1/2).
"""
import math

import numpy as np
from scipy import optimize

C_LIGHT = 2.99792458e10
KPC = 3.0856775814913673e21
MYR = 3.15576e13


def stromgren_radius(Ndot, nH, alpha_B):
    return (3.0 * Ndot / (4.0 * math.pi * alpha_B * nH * nH)) ** (1.0 / 3.0)


def t_rec(nH, alpha_B):
    return 1.0 / (nH * alpha_B)


def front_radius(t, rS, trec):
    """Infinite light speed law r_S (1 - exp(-t/t_rec))^(1/3)."""
    return rS * (1.0 - math.exp(-t / trec)) ** (1.0 / 3.0)


def front_radius_relativistic(t, rS, trec, c):
    """Solve w = q y - ln(1 - y^3) for y, q = r_S / (c t_rec), w = t / t_rec."""
    q = rS / (c * trec)
    w = t / trec
    g = lambda y: q * y - math.log(1.0 - y ** 3) - w  # noqa: E731
    hi = 1.0 - 1e-15
    if g(hi) < 0:
        return rS
    return rS * optimize.brentq(g, 0.0, hi, xtol=1e-15)


def photo_equilibrium_x(nH, alpha, beta, Gamma):
    """Root in [0,1] of n_H (alpha+beta) x^2 + (Gamma - beta n_H) x - Gamma = 0
    (H only, n_e = x n_H, constant photoionisation rate Gamma)."""
    a = nH * (alpha + beta)
    b = Gamma - beta * nH
    c = -Gamma
    disc = math.sqrt(b * b - 4.0 * a * c)
    # numerically stable root
    if b >= 0:
        return (2.0 * c) / (-b - disc)
    return (-b + disc) / (2.0 * a)


def ifront_radius(xHII, dx, corner=True, level=0.5):
    """Radius [cm] where the spherically averaged x_HII first drops below
    `level`; radii measured from the box corner (octant runs) or centre.
    Shells of width dx; linear interpolation between shell centres."""
    nz, ny, nx = xHII.shape
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    if corner:
        r = np.sqrt((i + 0.5) ** 2 + (j + 0.5) ** 2 + (k + 0.5) ** 2)
    else:
        r = np.sqrt((i + 0.5 - nx / 2) ** 2 + (j + 0.5 - ny / 2) ** 2 + (k + 0.5 - nz / 2) ** 2)
    nb = int(min(nx, ny, nz))
    b = np.floor(r).astype(int)
    prof = np.zeros(nb)
    for s in range(nb):
        m = b == s
        prof[s] = xHII[m].mean() if m.any() else np.nan
    rc = np.arange(nb) + 0.5
    for s in range(1, nb):
        if prof[s] < level <= prof[s - 1]:
            t = (prof[s - 1] - level) / (prof[s - 1] - prof[s])
            return (rc[s - 1] + t * (rc[s] - rc[s - 1])) * dx
    if prof[0] < level:
        return 0.0
    return nb * dx

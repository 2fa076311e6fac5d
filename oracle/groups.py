"""Oracle-side photon-group attributes (test infrastructure only).

Group cross sections and energies are inputs of the RT step (Sec. 2,
Eqs. (csn_multi), (egy_multi), (cse_multi)), averaged over a source spectrum
J(nu) within each frequency band, with the Verner et al. (1996) fits of the
appendix on cross sections (Eq. (PhI), table "Photoionization cross section
parameters") for sigma(eps).  This module integrates them for a blackbody by
adaptive quadrature (scipy.integrate.quad).

READING: the table prints epsilon_0 = 0.1361 eV for HeI, which gives the
non-physical sigma_HeI(24.59 eV) ~ 1.7e-23 cm^2; 13.61 eV gives the textbook
threshold value 7.4e-18 cm^2 and is used.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate

EV = 1.602176634e-12        # erg
K_B_EV = 8.617333262e-5     # eV / K
EPS_ION = (13.60, 24.59, 54.42)   # eV: HI, HeI, HeII thresholds

# Verner fit parameters: eps0 [eV], sigma0 [cm^2], P, ya, yw, y0, y1
VERNER = {
    "HI": (0.4298, 5.475e-14, 2.963, 32.88, 0.0, 0.0, 0.0),
    "HeI": (13.61, 9.492e-16, 3.188, 1.469, 2.039, 0.4434, 2.136),
    "HeII": (1.720, 1.369e-14, 2.963, 32.88, 0.0, 0.0, 0.0),
}
SPECIES = ("HI", "HeI", "HeII")


def sigma(species: str, eps: float) -> float:
    """Photoionisation cross section [cm^2] at photon energy eps [eV], Eq. (PhI)."""
    eth = EPS_ION[SPECIES.index(species)]
    if eps < eth:
        return 0.0
    e0, s0, P, ya, yw, y0, y1 = VERNER[species]
    x = eps / e0 - y0
    y = math.sqrt(x * x + y1 * y1)
    return s0 * ((x - 1.0) ** 2 + yw * yw) * y ** (0.5 * P - 5.5) / (1.0 + math.sqrt(y / ya)) ** P


def _planck_energy(eps: float, Tbb: float) -> float:
    """Blackbody spectral energy density J per unit energy, up to a constant."""
    x = eps / (K_B_EV * Tbb)
    if x > 700.0:
        return 0.0
    return eps ** 3 / math.expm1(x)


def _quad(fn, a, b):
    pts = [p for p in EPS_ION if a < p < b]
    if math.isinf(b):
        v1, _ = integrate.quad(fn, a, 2000.0, points=pts or None, limit=400, epsabs=0, epsrel=1e-13)
        v2, _ = integrate.quad(fn, 2000.0, np.inf, limit=200, epsabs=0, epsrel=1e-13)
        return v1 + v2
    v, _ = integrate.quad(fn, a, b, points=pts or None, limit=400, epsabs=0, epsrel=1e-13)
    return v


def group_attributes(bands, Tbb: float = 1e5):
    """Averages over each band [lo, hi) eV of a Tbb blackbody.

    Returns dict with sigN [G][3], sigE [G][3] (cm^2), egy [G] (erg) and the
    fraction of the ionising photons (eps >= bands[0][0]) in each band.
    """
    J = lambda e: _planck_energy(e, Tbb)            # noqa: E731
    Jn = lambda e: _planck_energy(e, Tbb) / e       # noqa: E731  photon number
    G = len(bands)
    sigN = np.zeros((G, 3))
    sigE = np.zeros((G, 3))
    egy = np.zeros(G)
    nphot = np.zeros(G)
    for i, (lo, hi) in enumerate(bands):
        n_int = _quad(Jn, lo, hi)
        e_int = _quad(J, lo, hi)
        nphot[i] = n_int
        egy[i] = e_int / n_int * EV
        for j, sp in enumerate(SPECIES):
            if hi <= EPS_ION[j]:
                continue   # band wholly below the threshold: sigma = 0 exactly
            sigN[i, j] = _quad(lambda e: sigma(sp, e) * Jn(e), lo, hi) / n_int
            sigE[i, j] = _quad(lambda e: sigma(sp, e) * J(e), lo, hi) / e_int
    total = _quad(Jn, bands[0][0], np.inf)
    return {"sigN": sigN, "sigE": sigE, "egy": egy, "photon_fraction": nphot / total}


THREE_BANDS = ((13.60, 24.59), (24.59, 54.42), (54.42, math.inf))
ONE_BAND = ((13.60, math.inf),)

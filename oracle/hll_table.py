"""Oracle-side table of the HLL wave speeds (test infrastructure only).

Sec. 3.2 of the paper takes lambda_min / lambda_max, the extreme eigenvalues
of the flux Jacobian dF/dU of the M1 system, from a table of Gonzalez et al.
(2007) as a function of the reduced flux f and of the angle between the flux
and the cell interface.  That table is not printed, so the oracle rebuilds
it (READING): for each (f, mu), mu = n . e_x, it forms the 4x4 Jacobian of
the x-direction flux

    F_x(U) = [F_x, P_xx, P_xy, P_xz],  P = N D(f, n)  (c = 1 units),

with D the Eddington tensor of Eqs. (eddTens), (Udir), by complex-step
differentiation, and takes its eigenvalues with LAPACK (numpy.linalg.eigvals).
The table is in units of c; the transport multiplies by the reduced light
speed.  Grid: f_k = k/(NF-1), mu_j = -1 + 2 j/(NMU-1); layout [NF][NMU][2]
with (lambda_min, lambda_max).  At f = 0 the direction is undefined and the
Jacobian is that of the isotropic closure, eigenvalues -1/sqrt(3), 0, 0,
+1/sqrt(3), for every mu.  At f = 1 the Jacobian is defective: all four
eigenvalues coalesce onto mu (the free-streaming speed across the face), so
a numerical eigensolver loses half its digits there; that row stores the
limit mu exactly.
"""
from __future__ import annotations

import functools

import numpy as np

NF = 257
NMU = 257
_H = 1e-30


def _xflux(U: np.ndarray) -> np.ndarray:
    """x-direction M1 flux of state U = (N, Fx, Fy, Fz), analytic in U."""
    N, Fx, Fy, Fz = U
    Fm = np.sqrt(Fx * Fx + Fy * Fy + Fz * Fz)
    f = Fm / N
    chi = (3.0 + 4.0 * f * f) / (5.0 + 2.0 * np.sqrt(4.0 - 3.0 * f * f))
    n = np.array([Fx, Fy, Fz]) / Fm
    a = 0.5 * (1.0 - chi)
    b = 0.5 * (3.0 * chi - 1.0)
    Pxx = N * (a + b * n[0] * n[0])
    Pxy = N * (b * n[0] * n[1])
    Pxz = N * (b * n[0] * n[2])
    return np.array([Fx, Pxx, Pxy, Pxz])


def jacobian(f: float, mu: float) -> np.ndarray:
    """dF_x/dU at N = 1, F = f (mu, sqrt(1-mu^2), 0), by complex step."""
    s = np.sqrt(max(0.0, 1.0 - mu * mu))
    U0 = np.array([1.0, f * mu, f * s, 0.0], dtype=np.complex128)
    J = np.zeros((4, 4))
    for k in range(4):
        U = U0.copy()
        U[k] += 1j * _H
        J[:, k] = np.imag(_xflux(U)) / _H
    return J


def eigen_extremes(f: float, mu: float) -> tuple[float, float]:
    if f == 0.0:
        r = 1.0 / np.sqrt(3.0)
        return -r, r
    if f == 1.0:
        return float(mu), float(mu)
    ev = np.linalg.eigvals(jacobian(f, mu))
    ev = np.real(ev)
    return float(ev.min()), float(ev.max())


@functools.lru_cache(maxsize=4)
def table(nf: int = NF, nmu: int = NMU) -> np.ndarray:
    t = np.zeros((nf, nmu, 2))
    for k in range(nf):
        f = k / (nf - 1)
        for j in range(nmu):
            mu = -1.0 + 2.0 * j / (nmu - 1)
            t[k, j] = eigen_extremes(f, mu)
    t.setflags(write=False)
    return t

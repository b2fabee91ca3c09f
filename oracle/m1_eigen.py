"""HLL wave speeds of the M1 system: eigenvalue table of the flux Jacobian.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests and ``bench.py``'s
CPU legs use it; the CUDA library builds its own table from its own derivation.

The HLL Riemann solver (Part III, "Riemann solvers", Eq. riemann-HLL) bounds the waves of
the local Riemann problem by the smallest and largest eigenvalue of the Jacobian
dF/dU of the M1 flux along the interface normal n.  The paper notes that the eigenvalues
depend only on the reduced flux f = |F|/(cE) and the angle theta between F and n, and that
they are tabulated over (theta, f) and interpolated rather than computed per interaction.

Here, with c = 1 and E = 1 (the eigenvalues scale with c and do not depend on E):
  * the flux along n = e_x is F_n(U) = (F . n, P(U) n) with the M1 pressure
    P = E [ (1 - chi)/2 I + (3 chi - 1)/2 F F^T / |F|^2 ],
    chi = (3 + 4 f^2) / (5 + 2 sqrt(4 - 3 f^2)) (Eq. eddington and the M1 closure);
  * its 4 x 4 Jacobian at U = (1, f cos theta, f sin theta, 0) is taken by complex-step
    differentiation (exact to rounding: no step-size error);
  * its eigenvalues come from numpy.linalg.eigvals; the table keeps the largest and the
    smallest (real parts; the imaginary parts vanish to rounding: the system is hyperbolic);
  * at f = 1 (free streaming) all four eigenvalues equal cos theta.  That quadruple root is
    entered as its exact value: a numerical eigen-solver scatters by ~1e-8 around it.

Grid (a reading: the paper does not give one): NF = 101 values of f = i/100 and NTH = 101
values of theta = j pi/100; lookups interpolate bilinearly in (f, theta).
"""
from __future__ import annotations

import numpy as np

NF = 101
NTH = 101


def _m1_flux_along_x(U):
    """(F . e_x, P e_x) for one state U = (E, Fx, Fy, Fz); complex-safe (no conjugation)."""
    E = U[0]
    F = U[1:]
    FF = F @ F
    f2 = FF / (E * E)
    chi = (3.0 + 4.0 * f2) / (5.0 + 2.0 * np.sqrt(4.0 - 3.0 * f2))
    n = np.array([1.0, 0.0, 0.0])
    P_n = E * (1.0 - chi) / 2.0 * n
    if FF != 0:
        # (3 chi - 1)/2 is of order f^2, so the direction term vanishes with F
        P_n = P_n + E * (3.0 * chi - 1.0) / 2.0 * F * (F @ n) / FF
    return np.concatenate([[F @ n], P_n])


def jacobian(f: float, theta: float, h: float = 1e-30) -> np.ndarray:
    """dF_n/dU at E = 1, F = f (cos theta, sin theta, 0), n = e_x, by complex steps."""
    U = np.array([1.0, f * np.cos(theta), f * np.sin(theta), 0.0])
    J = np.zeros((4, 4))
    for k in range(4):
        Uc = U.astype(complex)
        Uc[k] += 1j * h
        J[:, k] = np.imag(_m1_flux_along_x(Uc)) / h
    return J


def eigen_extremes(f: float, theta: float):
    """(largest, smallest) eigenvalue of the Jacobian, in units of c."""
    if f >= 1.0:
        return np.cos(theta), np.cos(theta)
    ev = np.linalg.eigvals(jacobian(f, theta)).real
    return ev.max(), ev.min()


def table(nf: int = NF, nth: int = NTH):
    """lmax, lmin: [nf, nth] arrays over f = i/(nf-1), theta = j pi/(nth-1)."""
    lmax = np.empty((nf, nth))
    lmin = np.empty((nf, nth))
    for i in range(nf):
        f = i / (nf - 1)
        for j in range(nth):
            lmax[i, j], lmin[i, j] = eigen_extremes(f, j * np.pi / (nth - 1))
    return lmax, lmin


_TABLE = None


def default_table():
    global _TABLE
    if _TABLE is None:
        _TABLE = table()
    return _TABLE

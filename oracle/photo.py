"""Photo-ionisation sink of the photon groups: cross sections, blackbody group averages and
photon-number to luminosity conversion.

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the tests and ``bench.py``'s CPU
legs use it; the CUDA library has its own host implementation.

Thesis passages (Part III):
  * photo-ionisation cross sections: the fit of Eq. sigma-parametrizaiton with the
    parameters of Table tab:cross-sections (H0, He0, He+), zero below the ionisation
    thresholds of Eqs. nuIonHI, nuIonHeI, nuIonHeII (13.60, 24.59, 54.42 eV);
  * group averages for an assumed blackbody spectrum (Eq. blackbody): the mean photon
    energy of a group and the number- and energy-weighted cross sections (Eqs. sigma_N,
    sigma_E);
  * the sink of every group: dE_i/dt = -sum_j n_j sigma^N_ij c E_i, and the same for F_i
    (Eqs. dEdt-group, dFdt-group);
  * Appendix "Converting Photon Number Emission Rates to Photon Energy Emission Rates":
    L_i = Ndot int_group J / int_{nu_min}^inf J/(h nu).

Readings: the table's sigma_0 is already in cm^2 (the "x 10^-18 cm^2" of the equation is
the megabarn convention of the fit's source; with it, sigma(H0, 13.6 eV) = 6.3e-18 cm^2,
the known threshold value).  Frequencies in Hz, energies in erg, CGS constants below.
Integrals by scipy.integrate.quad.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate

H_PLANCK = 6.62607015e-27      # erg s
K_BOLTZ = 1.380649e-16         # erg / K
EV = 1.602176634e-12           # erg

# Table tab:cross-sections: E0 [eV], sigma0 [cm^2], y_a, P, y_w, y_0, y_1
FIT = {
    "HI": (0.4298, 5.475e-14, 32.88, 2.963, 0.0, 0.0, 0.0),
    "HeI": (13.61, 9.492e-16, 1.469, 3.188, 2.039, 0.4434, 2.136),
    "HeII": (1.720, 1.369e-14, 32.88, 2.963, 0.0, 0.0, 0.0),
}
# ionisation energies, Eqs. nuIonHI, nuIonHeI, nuIonHeII [eV]
E_ION = {"HI": 13.60, "HeI": 24.59, "HeII": 54.42}
SPECIES = ("HI", "HeI", "HeII")


def cross_section(species: str, E_eV: float) -> float:
    """sigma(E) in cm^2 (Eq. sigma-parametrizaiton); zero below the threshold."""
    if E_eV < E_ION[species]:
        return 0.0
    E0, s0, ya, P, yw, y0, y1 = FIT[species]
    x = E_eV / E0 - y0
    y = math.sqrt(x * x + y1 * y1)
    F = ((x - 1.0) ** 2 + yw * yw) * y ** (0.5 * P - 5.5) * (1.0 + math.sqrt(y / ya)) ** (-P)
    return s0 * F


def blackbody(nu: float, T: float) -> float:
    """J_nu(T) up to its constant factor (Eq. blackbody): nu^3 / (exp(h nu / k T) - 1)."""
    return nu ** 3 / math.expm1(H_PLANCK * nu / (K_BOLTZ * T))


def _quad(f, a, b):
    # the spectrum falls as exp(-h nu / kT): beyond h nu = 700 kT it is below double range
    return integrate.quad(f, a, b, epsabs=0.0, epsrel=1e-12, limit=1000)[0]


def _upper(b, T):
    return min(b, 700.0 * K_BOLTZ * T / H_PLANCK)


def _split(a, b, T):
    """Integration breakpoints: the species thresholds inside (a, b) (the cross sections
    jump there)."""
    pts = [a]
    for s in SPECIES:
        nu = E_ION[s] * EV / H_PLANCK
        if a < nu < b:
            pts.append(nu)
    pts.append(b)
    return sorted(pts)


def group_averages(T: float, nu_edges):
    """(eps_mean [G] erg, sigma_N [G, 3] cm^2, sigma_E [G, 3] cm^2) for a blackbody of
    temperature T over the groups [nu_edges[i], nu_edges[i+1]) (the last edge may be inf)."""
    G = len(nu_edges) - 1
    eps = np.empty(G)
    sN = np.zeros((G, 3))
    sE = np.zeros((G, 3))
    for i in range(G):
        a, b = nu_edges[i], _upper(nu_edges[i + 1], T)
        pts = _split(a, b, T)
        segs = list(zip(pts[:-1], pts[1:]))
        e_int = sum(_quad(lambda nu: blackbody(nu, T), p, q) for p, q in segs)
        n_int = sum(_quad(lambda nu: blackbody(nu, T) / (H_PLANCK * nu), p, q) for p, q in segs)
        eps[i] = e_int / n_int
        for j, s in enumerate(SPECIES):
            sig = lambda nu: cross_section(s, H_PLANCK * nu / EV)
            sN[i, j] = sum(_quad(lambda nu: blackbody(nu, T) / (H_PLANCK * nu) * sig(nu), p, q)
                           for p, q in segs) / n_int
            sE[i, j] = sum(_quad(lambda nu: blackbody(nu, T) * sig(nu), p, q) for p, q in segs) / e_int
    return eps, sN, sE


def number_to_luminosity(T: float, Ndot: float, nu_edges):
    """L_i [erg/s] of the groups for an emission of Ndot photons/s above nu_edges[0]
    (Appendix "Converting Photon Number Emission Rates to Photon Energy Emission Rates")."""
    G = len(nu_edges) - 1
    top = _upper(math.inf, T)
    n_all = _quad(lambda nu: blackbody(nu, T) / (H_PLANCK * nu), nu_edges[0], top)
    return np.array([_quad(lambda nu: blackbody(nu, T), nu_edges[i], _upper(nu_edges[i + 1], T)) / n_all * Ndot
                     for i in range(G)])


def absorption(n_species, sigma_N):
    """alpha [G, N] = sum_j sigma_N[g, j] n_j (Eq. dEdt-group); n_species [3, N]."""
    return np.asarray(sigma_N) @ np.asarray(n_species)

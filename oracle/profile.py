"""FP64 oracle for the laterally averaged charge density rho(z) and potential psi(z) (Sec. II.C).

Test infrastructure: only tests/ use this module; the GPU library does not.

* rho(z): the charge per unit volume averaged over x and y on a uniform grid of nbins bins across
  the Ewald box in z (bin width h = L_z / nbins).  Electrolyte point charges fall into the bin that
  holds their wrapped z; an electrode site carries a Gaussian charge (Eq. 2), whose z-projection
  q eta / sqrt(pi) exp(-eta^2 (z - z_i)^2) is integrated over each bin (differences of erf,
  periodic images included).  Densities are per bin volume A h (A = L_x L_y).
* psi(z): the 1-D Poisson equation of Sec. II.C, d^2 psi / dz^2 = -rho / eps0, with 1 / eps0 =
  4 pi k_e, discretised by the periodic second difference on the bin centres and inverted as a
  matrix (the matrix method of Sec. II.C): the finite-difference matrix D is singular (constants),
  so it is bordered by the zero-mean condition, [[D, e], [e^T, 0]] [psi; lam] = [f; 0], whose
  unique solution is the zero-mean psi with D psi = f - lam e, lam = mean(f) (zero for a neutral
  cell).  Finite field: the charges' periodic
  potential plus the applied ramp dpsi z / L_z, so psi(L_z) - psi(0) = dpsi across the boundary;
  doubled cell and slab: continuity (the periodic solution itself).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

from .ewald import KE


def charge_density_z(box_z, area, nbins, elyt_z, elyt_q, elec_z, elec_q, eta) -> np.ndarray:
    """rho [nbins] in e / A^3 on bins of width box_z / nbins over [0, box_z).
    Sec. II.C; 0.34 A bins as in Appendix B."""
    h = box_z / nbins
    rho = np.zeros(nbins)
    zw = np.mod(np.asarray(elyt_z, np.float64), box_z)
    idx = np.minimum(nbins - 1, np.floor(zw / h).astype(int))
    np.add.at(rho, idx, np.asarray(elyt_q, np.float64))
    edges = np.arange(nbins + 1) * h
    for z, q in zip(np.mod(np.asarray(elec_z, np.float64), box_z), np.asarray(elec_q, np.float64)):
        for shift in (-box_z, 0.0, box_z):
            c = z + shift
            frac = 0.5 * (erf(eta * (edges[1:] - c)) - erf(eta * (edges[:-1] - c)))
            rho += q * frac
    return rho / (area * h)


def second_difference_matrix(nbins, h) -> np.ndarray:
    """Periodic (psi_{i+1} - 2 psi_i + psi_{i-1}) / h^2 as a dense matrix.
    Sec. II.C, Eq. 16 (low-order finite differences)."""
    D = -2.0 * np.eye(nbins) + np.eye(nbins, k=1) + np.eye(nbins, k=-1)
    D[0, -1] = D[-1, 0] = 1.0
    return D / (h * h)


def potential_z(rho, box_z, geometry="ff", dpsi=0.0) -> np.ndarray:
    """psi [nbins] in V at the bin centres (zero-mean periodic part, plus the finite-field ramp).
    Sec. II.C, Eq. 16 with the boundary condition of each geometry."""
    nbins = len(rho)
    h = box_z / nbins
    D = second_difference_matrix(nbins, h)
    M = np.zeros((nbins + 1, nbins + 1))
    M[:nbins, :nbins] = D
    M[:nbins, nbins] = 1.0
    M[nbins, :nbins] = 1.0
    rhs = np.zeros(nbins + 1)
    rhs[:nbins] = -4.0 * math.pi * KE * np.asarray(rho, np.float64)
    phi = np.linalg.solve(M, rhs)[:nbins]
    if geometry == "ff":
        z = (np.arange(nbins) + 0.5) * h
        phi = phi + dpsi * z / box_z
    return phi

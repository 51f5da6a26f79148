"""Analytical solution for a spherical molecule (radius d1, central charge q,
permittivity eps1) and a spherical surface (radius d2) of imposed potential
phi0 or charge sigma0, centres R apart, in a solvent (eps2, kappa) -- Section 4
(Eq. 18 (derivation1) to Eq. 44 (b_inf_dphi)), with the isolated-body limits of
Eq. 36 (a0_inf), Eq. 39-40 (energy_isolated_phi, b_inf_phi) and Eq. 43-44
(energy_isolated_dphi, b_inf_dphi).  Equation numbers follow the paper's LaTeX,
given with their labels.

Bessel functions: i_n(x) = sqrt(pi/2x) I_{n+1/2}(x), k_n(x) = sqrt(pi/2x)
K_{n+1/2}(x) (scipy.special.spherical_in / spherical_kn); the normalisation
of k_n cancels from every energy.  Reading G16: theta_1 and theta_2 are each
measured from the line of centres, pointing towards the other centre.
Reading G17: nu runs over 0..min(n, m) in Eq. 21 (Bnm).  Reading G14: the
factor (j+1) on the right of Eq. 25 (derivation4) multiplies delta_{0j} and is
dropped.  Reading G15: the imposed-charge system combines Eq. 25 (derivation4)
with Eq. 29 (derivation5_dphi), although the text names Eq. 26.
All quantities are in the oracle's internal units (units.py); energies are
returned in kcal/mol.
"""
import math

import numpy as np
from scipy.special import gammaln, spherical_in, spherical_kn

from .units import ENERGY_KCAL


def A_nu(n, m, nu):
    """A^nu_nm of Eq. 22 (Anm) (all factors positive; evaluated through log-gamma)."""
    lg = (gammaln(n - nu + 0.5) + gammaln(m - nu + 0.5) + gammaln(nu + 0.5)
          + gammaln(n + m - nu + 1) + math.log(n + m - 2 * nu + 0.5)
          - math.log(math.pi) - gammaln(m + n - nu + 1.5)
          - gammaln(n - nu + 1) - gammaln(m - nu + 1) - gammaln(nu + 1))
    return math.exp(lg)


def B_matrix(N, kR):
    """B_nm = sum_nu A^nu_nm k_{n+m-2nu}(kappa R), Eq. 21 (Bnm), for n, m < N."""
    B = np.zeros((N, N))
    for n in range(N):
        for m in range(N):
            B[n, m] = sum(A_nu(n, m, nu) * spherical_kn(n + m - 2 * nu, kR)
                          for nu in range(min(n, m) + 1))
    return B


def two_sphere(d1, d2, R, q, eps1, eps2, kappa, phi0=None, sigma0=None, N=40):
    """Coefficients (a_n, b_n) of Eq. 18 (derivation1) for the imposed-potential
    system Eq. 27-28 (system_phi, phi_terms) or the imposed-charge system
    Eq. 30-31 (system_dphi, dphi_terms), solved in the scaled unknowns A_n, B_n."""
    if (phi0 is None) == (sigma0 is None):
        raise ValueError("give exactly one of phi0, sigma0")
    n = np.arange(N)
    B = B_matrix(N, kappa * R)
    x1, x2 = kappa * d1, kappa * d2
    k1, k1p = spherical_kn(n, x1), spherical_kn(n, x1, derivative=True)
    i1, i1p = spherical_in(n, x1), spherical_in(n, x1, derivative=True)
    k2, k2p = spherical_kn(n, x2), spherical_kn(n, x2, derivative=True)
    i2, i2p = spherical_in(n, x2), spherical_in(n, x2, derivative=True)
    e_ratio = eps1 / eps2
    alpha = kappa * k1p - e_ratio * n / d1 * k1           # A_n = a_n * alpha_n
    j = n[:, None]
    Bnj = B.T                                            # [j, n] -> B_{n j}
    e0 = (n == 0).astype(float)
    rhs1 = -e_ratio * q / (4 * math.pi * eps1 * d1 ** 2) * e0
    if phi0 is not None:
        beta = k2                                        # B_n = b_n k_n(kd2)
        L = (2 * j + 1) * Bnj * (kappa * i1p[:, None] - e_ratio * j / d1 * i1[:, None]) / k2[None, :]
        M = (2 * j + 1) * Bnj * i2[:, None] / alpha[None, :]
        rhs2 = phi0 * e0
    else:
        beta = kappa * k2p                               # B_n = b_n kappa k_n'(kd2)
        L = (2 * j + 1) * Bnj * (i1p[:, None] / k2p[None, :] - e_ratio * j / d1 * i1[:, None] / (kappa * k2p[None, :]))
        M = (2 * j + 1) * Bnj * kappa * i2p[:, None] / alpha[None, :]
        rhs2 = -sigma0 / eps2 * e0
    I = np.eye(N)
    S = np.block([[I, L], [M, I]])
    sol = np.linalg.solve(S, np.concatenate([rhs1, rhs2]))
    a = sol[:N] / alpha
    b = sol[N:] / beta
    return a, b, B


def two_sphere_energies(d1, d2, R, q, eps1, eps2, kappa, phi0=None, sigma0=None, N=40):
    """Solvation (Eq. 32 energy_phi with Eq. 35 phi_reac_an2) and surface
    (Eq. 38 G_p_int / Eq. 42 G_c_int) energies of the
    interacting pair, in kcal/mol."""
    a, b, B = two_sphere(d1, d2, R, q, eps1, eps2, kappa, phi0, sigma0, N)
    x1, x2 = kappa * d1, kappa * d2
    phi_reac = (a[0] * spherical_kn(0, x1) + np.sum(b * B[:, 0]) * spherical_in(0, x1)
                - q / (4 * math.pi * eps1 * d1))
    solv = 0.5 * q * phi_reac
    if phi0 is not None:
        surf = 2 * math.pi * kappa * phi0 * d2 ** 2 * eps2 * (
            b[0] * spherical_kn(0, x2, derivative=True)
            + np.sum(a * B[:, 0]) * spherical_in(0, x2, derivative=True))
    else:
        surf = 2 * math.pi * sigma0 * d2 ** 2 * (
            b[0] * spherical_kn(0, x2) + np.sum(a * B[:, 0]) * spherical_in(0, x2))
    return float(solv) * ENERGY_KCAL, float(surf) * ENERGY_KCAL


def isolated_molecule_solvation(d1, q, eps1, eps2, kappa):
    """R -> infinity of Eq. 35 (phi_reac_an2) with a_0 from Eq. 36 (a0_inf) (kcal/mol)."""
    x1 = kappa * d1
    a0 = -q / d1 ** 2 * (eps1 / eps2) / (4 * math.pi * kappa * spherical_kn(0, x1, derivative=True) * eps1)
    phi_reac = a0 * spherical_kn(0, x1) - q / (4 * math.pi * eps1 * d1)
    return 0.5 * q * phi_reac * ENERGY_KCAL


def isolated_surface_potential(d2, phi0, eps2, kappa):
    """Eq. 39 (energy_isolated_phi) with b_0 from Eq. 40 (b_inf_phi) (kcal/mol)."""
    x2 = kappa * d2
    b0 = phi0 / spherical_kn(0, x2)
    return 2 * math.pi * kappa * phi0 * d2 ** 2 * b0 * spherical_kn(0, x2, derivative=True) * eps2 * ENERGY_KCAL


def isolated_surface_charge(d2, sigma0, eps2, kappa):
    """Eq. 43 (energy_isolated_dphi) with b_0 from Eq. 44 (b_inf_dphi) (kcal/mol)."""
    x2 = kappa * d2
    b0 = -sigma0 / (eps2 * kappa * spherical_kn(0, x2, derivative=True))
    return 2 * math.pi * sigma0 * d2 ** 2 * b0 * spherical_kn(0, x2) * ENERGY_KCAL


def interaction(d1, d2, R, q, eps1, eps2, kappa, phi0=None, sigma0=None, N=40):
    """F_int of Eq. 17 (interaction_energy) for the two-sphere system (kcal/mol); the single central
    charge has no Coulomb energy."""
    solv, surf = two_sphere_energies(d1, d2, R, q, eps1, eps2, kappa, phi0, sigma0, N)
    iso_m = isolated_molecule_solvation(d1, q, eps1, eps2, kappa)
    if phi0 is not None:
        iso_s = isolated_surface_potential(d2, phi0, eps2, kappa)
    else:
        iso_s = isolated_surface_charge(d2, sigma0, eps2, kappa)
    return (solv + surf) - (iso_m + iso_s), dict(solv=solv, surf=surf, iso_mol=iso_m, iso_surf=iso_s)

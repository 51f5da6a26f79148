"""Energies of Section 3.3 (Eq. 11-17), from a solution vector of the block
system, in kcal/mol.

  F_coul(a)  = 1/2 sum_{k != l} q_k q_l / (4 pi eps_a r_kl)              (Coulomb)
  phi_reac(r_k) = -K_L^{r_k}(phi_a) + V_L^{r_k}(dphi_a)                  (Eq. 13)
  F_solv(a)  = 1/2 sum_k q_k phi_reac(r_k)     (Eq. 11-12; reading G1 keeps
               the 1/2 of Eq. 11, as Eq. 32 (energy_phi) of Section 4 does)
  F_surf(s)  = 1/2 sum_j phi_j sigma0 A_j       imposed charge (Eq. 15)
             = -1/2 sum_j phi0 sigma_j A_j      imposed potential, with
               sigma_j = -eps_out dphi_j/dn (reading G3, the sign of Eq. 1)
  F_total    = F_coul + F_surf + F_solv                                   (Eq. 16)
  F_int      = F_total(assembly) - sum_i F_total(body i alone)            (Eq. 17)
phi_reac uses the same three tiers as the matrix entries, with r_k as the
target (reading G11).
"""
import numpy as np

from .bem import DIELECTRIC, SET_CHARGE, System
from .integrals import panel_operator_blocks
from .units import ENERGY_KCAL


def reaction_potential(sys: System, x, a):
    b = sys.bodies[a]
    xq = b.world_charges()
    if len(xq) == 0:
        return np.zeros(0)
    phi, dphi = sys.blocks(x, a)
    VL, KL, _, _ = panel_operator_blocks(xq, sys.panels[a], sys.kappa, sys.p.K,
                                         sys.p.K_near, sys.p.n_edge, None)
    return -KL @ phi + VL @ dphi


def coulomb_energy(b, xq=None):
    xq = b.world_charges() if xq is None else xq
    q = b.charge_q
    if len(q) < 2:
        return 0.0
    d = xq[:, None, :] - xq[None, :, :]
    r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
    np.fill_diagonal(r, np.inf)
    return 0.5 * float((q[:, None] * q[None, :] / (4 * np.pi * b.eps_in * r)).sum()) * ENERGY_KCAL


def energies(sys: System, x):
    """dict with coulomb, solvation, surface, total (kcal/mol), summed over bodies,
    plus per-body lists."""
    out = {"coulomb": 0.0, "solvation": 0.0, "surface": 0.0, "per_body": []}
    for a, b in enumerate(sys.bodies):
        e = {"coulomb": 0.0, "solvation": 0.0, "surface": 0.0}
        if b.kind == DIELECTRIC:
            e["coulomb"] = coulomb_energy(b)
            pr = reaction_potential(sys, x, a)
            e["solvation"] = 0.5 * float(b.charge_q @ pr) * ENERGY_KCAL
        else:
            (u,) = sys.blocks(x, a)
            A = sys.panels[a].A
            if b.kind == SET_CHARGE:
                e["surface"] = 0.5 * float(np.sum(u * b.bc_value * A)) * ENERGY_KCAL
            else:
                sigma = -sys.eps_out * u
                e["surface"] = -0.5 * float(np.sum(b.bc_value * sigma * A)) * ENERGY_KCAL
        for k in ("coulomb", "solvation", "surface"):
            out[k] += e[k]
        e["total"] = e["coulomb"] + e["solvation"] + e["surface"]
        out["per_body"].append(e)
    out["total"] = out["coulomb"] + out["solvation"] + out["surface"]
    return out


def interaction_energy(total_assembly, totals_isolated):
    """Eq. 17."""
    return total_assembly - sum(totals_isolated)

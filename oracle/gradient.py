"""Gradients of the total free energy (Eq. 16) by the discrete adjoint,
dense and FP64.  The paper has no gradient; this restates the adjoint method
for the system of Eq. 6 / Eq. 7 so that the CUDA gradients can be checked.

x solves A(t) x = b(q, bc, t); F(x, q, bc) = F_coul(q) + F_solv(x, q) +
F_surf(x, bc) with
  F_solv = 1/2 q . phi_reac,  phi_reac = C x  (Eq. 13, charge rows of -K_L, V_L)
  F_surf = 1/2 beta sum_j A_j u_j,  beta = sigma0 (imposed charge) or
           eps_out phi0 (imposed potential)  (Eq. 15 with reading G3).
Adjoint: A^T lam = dF/dx; then dF/dp = dF/dp|_x + lam . (db/dp - dA/dp x).
  q_k:  Coulomb potential of the other charges + 1/2 phi_reac(r_k)
        + (1/eps_a) sum_{interior rows i} lam_i / (4 pi |c_i - r_k|)
  bc:   1/2 (beta/bc) sum A_j u_j + lam . b_known(bc = 1)
  t_m (translation of body m): only the Yukawa cross-body terms of the
        exterior and surface rows depend on t; with U^(b) the combined
        potential of body b's full (unknown + imposed) densities,
        dF/dt_m = -[ sum_{rows i of m} lam_i grad U^(b != m)(c_i)
                    - sum_{rows i not of m} lam_i grad U^(m)(c_i) ].
  The cross-body entries use the K-point rule only (bodies farther apart
  than 2L; reading G20).
Units: energies kcal/mol; dF/dq per e; dF/dsigma0 per C/m^2; dF/dphi0 per V;
dF/dt per Angstrom.
"""
import math

import numpy as np
import scipy.linalg

from .bem import DIELECTRIC, SET_CHARGE, System
from .energy import energies
from .integrals import panel_operator_blocks
from .units import ENERGY_KCAL, phi_from_volt, sigma_from_c_m2

FOUR_PI = 4.0 * math.pi


def _full_densities(sys, x, b):
    """Single- and double-layer densities (psi_Y, phi_Y) of body b with the
    imposed parts included."""
    bb = sys.bodies[b]
    if bb.kind == DIELECTRIC:
        phi, dphi = sys.blocks(x, b)
        return (bb.eps_in / sys.eps_out) * dphi, phi
    (u,) = sys.blocks(x, b)
    N = sys.panels[b].N
    if bb.kind == SET_CHARGE:
        return np.full(N, -bb.bc_value / sys.eps_out), u
    return u, np.full(N, bb.bc_value)


def yukawa_gradient(sys, targets, b, psi, phi):
    """grad_x of U_Y(x) = sum_s w_s [psi G_Y(x - y_s) - phi n.grad_y G_Y(x - y_s)]
    over body b's K-point nodes (no near tier), targets (T,3) -> (T,3)."""
    pn = sys.panels[b]
    y, w = pn.points(sys.p.K)
    y = y.reshape(-1, 3)
    q = (w * psi[:, None]).reshape(-1)
    p = ((w * phi[:, None])[..., None] * pn.n[:, None, :]).reshape(-1, 3)
    k = sys.kappa
    out = np.zeros((len(targets), 3))
    for t0 in range(0, len(targets), 64):
        d = targets[t0:t0 + 64, None, :] - y[None, :, :]
        r2 = np.einsum("tsk,tsk->ts", d, d)
        r = np.sqrt(r2)
        e = np.exp(-k * r)
        # grad of G_Y = e/(4 pi r): -(1 + k r) e d / (4 pi r^3)
        gG = -((1 + k * r) * e / r ** 3)[..., None] * d
        # grad of n.grad_y G_Y = p.d (1 + k r) e / (4 pi r^3) with p for n
        pd = np.einsum("sk,tsk->ts", p, d)
        f1 = (1 + k * r) * e / r ** 3
        f2 = (k * k * r2 + 3 * k * r + 3) * e / r ** 5
        gK = f1[..., None] * p[None, :, :] - (f2 * pd)[..., None] * d
        out[t0:t0 + 64] = (np.einsum("ts,tsk->tk", q[None, :] * np.ones_like(r), gG) - gK.sum(1)) / FOUR_PI
    return out


def gradients(sys: System):
    """dict: energies (oracle.energy.energies of the solution), dq (list per
    body, arrays), dbc (per body, None for molecules), dt (per body, (3,))."""
    A, rhs = sys.assemble()
    lu = scipy.linalg.lu_factor(A)
    x = scipy.linalg.lu_solve(lu, rhs)
    g = np.zeros(sys.n)
    nb = len(sys.bodies)
    phireac = [None] * nb
    for a, ba in enumerate(sys.bodies):
        o = sys.offsets[a]
        N = sys.panels[a].N
        if ba.kind == DIELECTRIC and len(ba.charge_q):
            xq = ba.world_charges()
            VL, KL, _, _ = panel_operator_blocks(xq, sys.panels[a], sys.kappa, sys.p.K, sys.p.K_near,
                                                 sys.p.n_edge, None)
            phi, dphi = sys.blocks(x, a)
            phireac[a] = -KL @ phi + VL @ dphi
            g[o:o + N] += -0.5 * (ba.charge_q @ KL)
            g[o + N:o + 2 * N] += 0.5 * (ba.charge_q @ VL)
        elif ba.kind != DIELECTRIC:
            beta = ba.bc_value if ba.kind == SET_CHARGE else sys.eps_out * ba.bc_value
            g[o:o + N] += 0.5 * beta * sys.panels[a].A
    lam = scipy.linalg.lu_solve(lu, g, trans=1)
    out = {"energies": energies(sys, x), "dq": [], "dbc": [], "dt": [], "x": x, "lam": lam}
    for a, ba in enumerate(sys.bodies):
        o = sys.offsets[a]
        N = sys.panels[a].N
        if ba.kind == DIELECTRIC:
            xq = ba.world_charges()
            q = ba.charge_q
            dq = np.zeros(len(q))
            if len(q):
                d = xq[:, None, :] - xq[None, :, :]
                r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
                np.fill_diagonal(r, np.inf)
                dq += (q[None, :] / (FOUR_PI * ba.eps_in * r)).sum(1)
                dq += 0.5 * phireac[a]
                dc = sys.panels[a].c[:, None, :] - xq[None, :, :]
                rc = np.sqrt(np.einsum("ijk,ijk->ij", dc, dc))
                dq += (lam[o:o + N] @ (1.0 / (FOUR_PI * rc))) / ba.eps_in
            out["dq"].append(dq * ENERGY_KCAL)
            out["dbc"].append(None)
        else:
            (u,) = sys.blocks(x, a)
            Aj = sys.panels[a].A
            # b_known for unit bc: the imposed terms of Eq. 6/7 are linear in bc
            saved = ba.bc_value
            ba.bc_value = 1.0
            _, rhs1 = sys.assemble()
            ba.bc_value = saved
            for a2, b2 in enumerate(sys.bodies):  # keep only the imposed parts
                if b2.kind == DIELECTRIC:
                    rhs1[sys.offsets[a2]:sys.offsets[a2] + sys.panels[a2].N] = 0.0
            for a2, b2 in enumerate(sys.bodies):
                if a2 != a and b2.kind != DIELECTRIC:
                    raise NotImplementedError("one imposed surface per system")
            fac = 1.0 if ba.kind == SET_CHARGE else sys.eps_out
            dbc = 0.5 * fac * float(u @ Aj) + float(lam @ rhs1)
            conv = sigma_from_c_m2(1.0) if ba.kind == SET_CHARGE else phi_from_volt(1.0)
            out["dq"].append(None)
            out["dbc"].append(dbc * conv * ENERGY_KCAL)
    # translations
    dens = [_full_densities(sys, x, b) for b in range(nb)]
    for m in range(nb):
        tot = np.zeros(3)
        for a, ba in enumerate(sys.bodies):
            o = sys.offsets[a]
            N = sys.panels[a].N
            lam_y = lam[o + N:o + 2 * N] if ba.kind == DIELECTRIC else lam[o:o + N]
            c = sys.panels[a].c
            for b in range(nb):
                if b == a:
                    continue
                if a == m:
                    tot -= lam_y @ yukawa_gradient(sys, c, b, *dens[b])
                elif b == m:
                    tot += lam_y @ yukawa_gradient(sys, c, m, *dens[m])
        out["dt"].append(tot * ENERGY_KCAL)
    return out

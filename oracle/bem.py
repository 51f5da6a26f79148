"""Dense boundary-element system of the paper (Section 2, Eq. 5-7), assembled
entry by entry with the three-tier integrals of Section 3.1, solved by LU.

Bodies are kept in a list.  A *dielectric* body (a molecule, interface Gamma_1)
carries unknowns [phi (N), dphi/dn (N)] (the interior values) and its point
charges; a *surface* body (Gamma_2) carries one unknown block u (N): dphi/dn
for imposed potential (Eq. 6) or phi for imposed charge (Eq. 7).  For one
molecule and one surface this is exactly Eq. 6 / Eq. 7; for one molecule alone
it is their upper-left 2x2 block.  With several bodies the same rows are
repeated per body, the multi-surface extension the paper mentions after Eq. 7.

Row blocks (normals out of every body into the solvent, reading G4):
  interior row of dielectric a (first line of Eq. 5):
      (1/2 + K_L^{aa}) phi_a - V_L^{aa} dphi_a = (1/eps_a) sum_k q_k/(4 pi |x - r_k|)
      (reading G2: the 1/eps_1 of Eq. 5 is kept on the right-hand side of Eq. 6/7)
  exterior row of dielectric a / row of surface s (second and third lines):
      sum_b [ delta_ab/2 phi_b - K_Y^{.b} phi_b + (eps_b/eps_out) V_Y^{.b} dphi_b ]
    + sum_t [ imposed potential: V_Y^{.t} u_t  (+ known -K_Y^{.t} phi0 + delta/2 phi0)
              imposed charge:    (delta/2 - K_Y^{.t}) u_t (+ known V_Y^{.t} dphi_t) ] = 0
  with dphi_t = -sigma0/eps_out on an imposed-charge surface (Eq. 1), and the
  known parts moved to the right-hand side.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg

from .geometry import Panels, rigid_transform
from .integrals import panel_operator_blocks

DIELECTRIC, SET_CHARGE, SET_POTENTIAL = 0, 1, 2


@dataclass
class Body:
    kind: int
    verts: np.ndarray
    tris: np.ndarray
    eps_in: float = 1.0
    charge_xyz: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    charge_q: np.ndarray = field(default_factory=lambda: np.zeros(0))
    bc_value: float = 0.0          # sigma0 (e/A^2) or phi0 (e/(eps0 A)) for surfaces
    R: np.ndarray = None           # rigid pose (world = R body + t)
    t: np.ndarray = None

    def world(self):
        return rigid_transform(self.verts, self.R, self.t)

    def world_charges(self):
        if len(self.charge_q) == 0:
            return np.zeros((0, 3))
        return rigid_transform(self.charge_xyz, self.R, self.t)

    @property
    def nunk(self):
        return 2 * len(self.tris) if self.kind == DIELECTRIC else len(self.tris)


@dataclass
class Params:
    K: int = 7            # far rule points (Section 3.1)
    K_near: int = 19      # fine rule points
    n_edge: int = 9       # Gauss points per edge, self integral
    theta: float = 0.5    # multipole acceptance (Section 3.2)
    P: int = 6            # Taylor order
    leaf_size: int = 32   # N_crit
    group_size: int = 32  # targets per interaction list


class System:
    """All bodies of one problem plus the solvent (eps_out, kappa)."""

    def __init__(self, bodies, eps_out, kappa, params=None):
        self.bodies = list(bodies)
        self.eps_out = float(eps_out)
        self.kappa = float(kappa)
        self.p = params or Params()
        self.panels = [Panels(b.world(), b.tris) for b in self.bodies]
        self.offsets = np.cumsum([0] + [b.nunk for b in self.bodies])
        self.n = int(self.offsets[-1])

    # ---- layout helpers -------------------------------------------------
    def blocks(self, x, a):
        """Views of the unknown blocks of body a in vector x."""
        o = self.offsets[a]
        N = self.panels[a].N
        if self.bodies[a].kind == DIELECTRIC:
            return x[o:o + N], x[o + N:o + 2 * N]
        return (x[o:o + N],)

    def operator_blocks(self, a, b, laplace):
        """V_L, K_L, V_Y, K_Y with targets = centroids of body a, sources = panels of b."""
        si = np.arange(self.panels[a].N) if a == b else None
        return panel_operator_blocks(self.panels[a].c, self.panels[b], self.kappa,
                                     self.p.K, self.p.K_near, self.p.n_edge, si, laplace)

    # ---- dense assembly (Eq. 6 / Eq. 7) ---------------------------------
    def assemble(self):
        """Dense matrix A (n x n) and right-hand side b of the block system."""
        idx, A, rhs = self.assemble_rows([np.arange(pn.N) for pn in self.panels])
        Af = np.zeros((self.n, self.n))
        bf = np.zeros(self.n)
        Af[idx] = A
        bf[idx] = rhs
        return Af, bf

    def assemble_rows(self, rows):
        """The rows of the dense system that belong to the target panels
        rows[a] (indices into body a's panels) of every body a: returns the
        global row indices, those rows of A and of the right-hand side.  The
        entries are those of assemble(); splitting the targets into chunks
        splits the assembly (the oracle's CPU timing runs chunks in parallel)."""
        idx, blocks, rhs_parts = [], [], []
        for a, ba in enumerate(self.bodies):
            ra = np.asarray(rows[a], dtype=np.int64)
            if len(ra) == 0:
                continue
            nr = len(ra)
            oa = self.offsets[a]
            Na = self.panels[a].N
            ext = oa + Na if ba.kind == DIELECTRIC else oa   # exterior/surface row start
            n_blk = 2 if ba.kind == DIELECTRIC else 1
            A = np.zeros((n_blk * nr, self.n))
            rhs = np.zeros(n_blk * nr)
            e0 = nr if ba.kind == DIELECTRIC else 0          # exterior/surface rows within A
            for b, bb in enumerate(self.bodies):
                Nb = self.panels[b].N
                ob = self.offsets[b]
                si = ra if a == b else None
                VL, KL, VY, KY = panel_operator_blocks(self.panels[a].c[ra], self.panels[b], self.kappa,
                                                       self.p.K, self.p.K_near, self.p.n_edge, si, a == b)
                if a == b:
                    I = np.zeros((nr, Nb))
                    I[np.arange(nr), ra] = 1.0
                else:
                    I = None
                if bb.kind == DIELECTRIC:
                    if a == b:   # interior row (Laplace), Eq. 5 line 1
                        A[0:nr, ob:ob + Nb] = 0.5 * I + KL
                        A[0:nr, ob + Nb:ob + 2 * Nb] = -VL
                    blk = -KY + (0.5 * I if a == b else 0.0)
                    A[e0:e0 + nr, ob:ob + Nb] = blk
                    A[e0:e0 + nr, ob + Nb:ob + 2 * Nb] = (bb.eps_in / self.eps_out) * VY
                elif bb.kind == SET_POTENTIAL:
                    phi0 = bb.bc_value
                    A[e0:e0 + nr, ob:ob + Nb] = VY
                    known = (-KY + (0.5 * I if a == b else 0.0)) @ np.full(Nb, phi0)
                    rhs[e0:e0 + nr] -= known
                else:            # SET_CHARGE
                    dphi = -bb.bc_value / self.eps_out
                    A[e0:e0 + nr, ob:ob + Nb] = -KY + (0.5 * I if a == b else 0.0)
                    rhs[e0:e0 + nr] -= VY @ np.full(Nb, dphi)
            if ba.kind == DIELECTRIC:
                rhs[0:nr] = self.coulomb_rhs(a)[ra]
                idx.append(oa + ra)
            idx.append(ext + ra)
            blocks.append(A)
            rhs_parts.append(rhs)
        return np.concatenate(idx), np.concatenate(blocks), np.concatenate(rhs_parts)

    def coulomb_rhs(self, a):
        """(1/eps_a) sum_k q_k / (4 pi |c_i - r_k|) at the centroids of body a (Eq. 5, G2)."""
        b = self.bodies[a]
        xq = b.world_charges()
        if len(xq) == 0:
            return np.zeros(self.panels[a].N)
        d = self.panels[a].c[:, None, :] - xq[None, :, :]
        r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
        return (b.charge_q[None, :] / (4 * np.pi * r)).sum(1) / b.eps_in

    def solve(self):
        """LU solve of the dense system (Section 3.2 replaces this by GMRES)."""
        A, rhs = self.assemble()
        lu = scipy.linalg.lu_factor(A)
        return scipy.linalg.lu_solve(lu, rhs)

    # ---- matrix-free application -----------------------------------------
    def densities(self, x, b):
        """Source densities of body b for the combined potential U = S_V - S_K:
        (psi_L, phi_L, psi_Y, phi_Y) per panel (see the module doc)."""
        bb = self.bodies[b]
        N = self.panels[b].N
        z = np.zeros(N)
        if bb.kind == DIELECTRIC:
            phi, dphi = self.blocks(x, b)
            return dphi, phi, (bb.eps_in / self.eps_out) * dphi, phi
        (u,) = self.blocks(x, b)
        if bb.kind == SET_POTENTIAL:
            return z, z, u, z
        return z, z, z, u

    def apply_rows(self, x, a, rows=None):
        """Direct-sum rows of A x for targets `rows` (indices into body a's
        panels; all when None), evaluated panel by panel with the same tiered
        entries as assemble() but without storing the matrix.  Returns the
        list of row-block values for body a (2 blocks for a dielectric)."""
        pa = self.panels[a]
        rows = np.arange(pa.N) if rows is None else np.asarray(rows)
        UL = np.zeros(len(rows))
        UY = np.zeros(len(rows))
        for b, bb in enumerate(self.bodies):
            psiL, phiL, psiY, phiY = self.densities(x, b)
            si = rows if a == b else None
            VL, KL, VY, KY = panel_operator_blocks(pa.c[rows], self.panels[b], self.kappa,
                                                   self.p.K, self.p.K_near, self.p.n_edge, si)
            if a == b and bb.kind == DIELECTRIC:
                UL += VL @ psiL - KL @ phiL
            UY += VY @ psiY - KY @ phiY
        ba = self.bodies[a]
        if ba.kind == DIELECTRIC:
            phi, dphi = self.blocks(x, a)
            return [0.5 * phi[rows] - UL, 0.5 * phi[rows] + UY]
        (u,) = self.blocks(x, a)
        if ba.kind == SET_CHARGE:
            return [UY + 0.5 * u[rows]]
        return [UY]

    def apply(self, x):
        """Full direct-sum product A x (same as assemble()[0] @ x)."""
        out = np.zeros(self.n)
        for a, ba in enumerate(self.bodies):
            o = self.offsets[a]
            N = self.panels[a].N
            for k, blk in enumerate(self.apply_rows(x, a)):
                out[o + k * N:o + (k + 1) * N] = blk
        return out

"""More interfaces (Section 2, after Eq. 7: Stern layers and solvent-filled
cavities are further surfaces whose equations add block rows), written out
region by region.  TEST INFRASTRUCTURE ONLY (see the package docstring).

Reading (the paper states the extension in one sentence and defers to its
multi-surface references; the rows below are Green's representation formula
applied in every region, in the notation of Eq. 5):

* Regions are the solvent (permittivity eps_out, screening kappa) and the
  interior of every dielectric body b (eps_in(b), kappa_in(b), 0 by default).
  Each body b lies in an outer region: the solvent, or the interior of its
  parent body p(b).  A Stern layer around a molecule M is a dielectric body S
  with eps_in(S) = eps_out and kappa_in(S) = 0 that is M's parent; a cavity C
  in M is a dielectric body with parent M (eps_in(C) = eps_out for solvent).
* Unknowns as in Eq. 6/7: a dielectric body carries phi and dphi/dn on its
  inner side (normals point from the body into its outer region); a surface
  with an imposed value carries one block (reading of Eq. 6/7) and bounds its
  outer region only.
* Region R is bounded by the bodies whose inner region is R (sign s = +1,
  inner-side density psi = dphi) and by the bodies whose outer region is R
  (s = -1, psi = (eps_in(b) / eps_R) dphi for a dielectric body, the block u
  of Eq. 6 or the imposed -sigma0 / eps_R of Eq. 7 for a surface), since the
  flux eps dphi/dn is continuous across a dielectric interface (Eq. 2).
  At a collocation point x on a body a bounding R:
      1/2 phi(x) - sum_{b bounds R} s_b [ V_R psi_b - K_R phi_b ](x)
          = (1/eps_R) sum_{k in R} q_k / (4 pi |x - r_k|)
  with V_R, K_R the Laplace (kappa_R = 0) or Yukawa (kappa_R) operators of
  Eq. 9 and the three-tier rules of Section 3.1.  A dielectric body has one
  such row for its inner and one for its outer region; a surface one for its
  outer region.  With every body in the solvent these are exactly the rows
  of Eq. 6/7 (System.assemble), which tests/test_oracle_regions.py checks.
* Solvation energy (Eq. 11-13): phi_reac(r_k) at a charge of body M is the
  representation in M's interior without the Coulomb term,
      phi_reac(r_k) = sum_{b bounds int(M)} s_b [ V psi_b - K phi_b ](r_k),
  i.e. M's own panels and those of its cavities.
"""
import numpy as np
import scipy.linalg

from .bem import DIELECTRIC, SET_CHARGE, SET_POTENTIAL, Params
from .energy import coulomb_energy
from .geometry import Panels
from .integrals import panel_operator_blocks
from .units import ENERGY_KCAL


class RegionSystem:
    """Bodies (oracle.bem.Body) with a parent per body (-1: the solvent) and
    the screening of each dielectric body's interior."""

    def __init__(self, bodies, eps_out, kappa, parent=None, kappa_in=None, params=None):
        self.bodies = list(bodies)
        nb = len(self.bodies)
        self.parent = list(parent) if parent is not None else [-1] * nb
        self.kappa_in = list(kappa_in) if kappa_in is not None else [0.0] * nb
        self.eps_out = float(eps_out)
        self.kappa = float(kappa)
        self.p = params or Params()
        for b, pb in enumerate(self.parent):
            if pb >= 0 and self.bodies[pb].kind != DIELECTRIC:
                raise ValueError("a parent must be a dielectric body")
            if pb == b:
                raise ValueError("a body cannot be its own parent")
        self.panels = [Panels(b.world(), b.tris) for b in self.bodies]
        self.offsets = np.cumsum([0] + [b.nunk for b in self.bodies])
        self.n = int(self.offsets[-1])

    # ---- regions: 0 = solvent, b + 1 = interior of dielectric body b
    def inner(self, b):
        return b + 1 if self.bodies[b].kind == DIELECTRIC else None

    def outer(self, b):
        return 0 if self.parent[b] < 0 else self.parent[b] + 1

    def region_eps(self, R):
        return self.eps_out if R == 0 else self.bodies[R - 1].eps_in

    def region_kappa(self, R):
        return self.kappa if R == 0 else self.kappa_in[R - 1]

    def boundary(self, R):
        """[(body, sign)] of the bodies bounding region R."""
        out = []
        for b in range(len(self.bodies)):
            if self.inner(b) == R:
                out.append((b, +1))
            elif self.outer(b) == R:
                out.append((b, -1))
        return out

    def rows(self, a):
        """[(row offset, region)] of body a's equations."""
        o = self.offsets[a]
        if self.bodies[a].kind == DIELECTRIC:
            return [(o, self.inner(a)), (o + self.panels[a].N, self.outer(a))]
        return [(o, self.outer(a))]

    def blocks(self, x, a):
        o = self.offsets[a]
        N = self.panels[a].N
        if self.bodies[a].kind == DIELECTRIC:
            return x[o:o + N], x[o + N:o + 2 * N]
        return (x[o:o + N],)

    def _vk(self, targets, b, kappa, self_index):
        VL, KL, VY, KY = panel_operator_blocks(targets, self.panels[b], kappa, self.p.K, self.p.K_near,
                                               self.p.n_edge, self_index)
        return (VY, KY) if kappa > 0 else (VL, KL)

    def assemble(self):
        """Dense matrix and right-hand side of all rows."""
        A = np.zeros((self.n, self.n))
        rhs = np.zeros(self.n)
        for a, ba in enumerate(self.bodies):
            Na = self.panels[a].N
            oa = self.offsets[a]
            for r0, R in self.rows(a):
                epsR, kapR = self.region_eps(R), self.region_kappa(R)
                # jump term of the unknown (or imposed) phi of body a
                if ba.kind == DIELECTRIC or ba.kind == SET_CHARGE:
                    A[r0:r0 + Na, oa:oa + Na] += 0.5 * np.eye(Na)
                else:
                    rhs[r0:r0 + Na] -= 0.5 * ba.bc_value
                for b, s in self.boundary(R):
                    bb = self.bodies[b]
                    Nb = self.panels[b].N
                    ob = self.offsets[b]
                    si = np.arange(Na) if a == b else None
                    V, K = self._vk(self.panels[a].c, b, kapR, si)
                    # row += -s (V psi - K phi)
                    if bb.kind == DIELECTRIC:
                        A[r0:r0 + Na, ob:ob + Nb] += s * K
                        f = 1.0 if s > 0 else bb.eps_in / epsR
                        A[r0:r0 + Na, ob + Nb:ob + 2 * Nb] += -s * f * V
                    elif bb.kind == SET_POTENTIAL:
                        A[r0:r0 + Na, ob:ob + Nb] += -s * V
                        rhs[r0:r0 + Na] -= s * K @ np.full(Nb, bb.bc_value)
                    else:
                        A[r0:r0 + Na, ob:ob + Nb] += s * K
                        psi = -bb.bc_value / epsR
                        rhs[r0:r0 + Na] += s * V @ np.full(Nb, psi)
                rhs[r0:r0 + Na] += self.coulomb(a, R)
        return A, rhs

    def charges_in(self, R):
        """(positions, charges) of the point charges in region R."""
        if R == 0:
            return np.zeros((0, 3)), np.zeros(0)
        b = self.bodies[R - 1]
        return b.world_charges(), b.charge_q

    def coulomb(self, a, R):
        xq, q = self.charges_in(R)
        if len(q) == 0:
            return np.zeros(self.panels[a].N)
        d = self.panels[a].c[:, None, :] - xq[None, :, :]
        r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
        return (q[None, :] / (4 * np.pi * r)).sum(1) / self.region_eps(R)

    def solve(self):
        A, rhs = self.assemble()
        return scipy.linalg.lu_solve(scipy.linalg.lu_factor(A), rhs)

    def reaction_potential(self, x, m):
        """phi_reac at the charges of dielectric body m (see the module doc)."""
        bm = self.bodies[m]
        xq = bm.world_charges()
        if len(xq) == 0:
            return np.zeros(0)
        R = self.inner(m)
        out = np.zeros(len(xq))
        for b, s in self.boundary(R):
            bb = self.bodies[b]
            V, K = self._vk(xq, b, self.region_kappa(R), None)
            if bb.kind == DIELECTRIC:
                phi, dphi = self.blocks(x, b)
                psi = dphi if s > 0 else (bb.eps_in / self.region_eps(R)) * dphi
            elif bb.kind == SET_POTENTIAL:
                (psi,) = self.blocks(x, b)
                phi = np.full(self.panels[b].N, bb.bc_value)
            else:
                (phi,) = self.blocks(x, b)
                psi = np.full(self.panels[b].N, -bb.bc_value / self.region_eps(R))
            out += s * (V @ psi - K @ phi)
        return out

    def energies(self, x):
        """coulomb, solvation, surface, total (kcal/mol) as oracle.energy.energies."""
        e = {"coulomb": 0.0, "solvation": 0.0, "surface": 0.0}
        for a, b in enumerate(self.bodies):
            if b.kind == DIELECTRIC:
                if len(b.charge_q):
                    e["coulomb"] += coulomb_energy(b)
                    e["solvation"] += 0.5 * float(b.charge_q @ self.reaction_potential(x, a)) * ENERGY_KCAL
            else:
                (u,) = self.blocks(x, a)
                A = self.panels[a].A
                if b.kind == SET_CHARGE:
                    e["surface"] += 0.5 * float(np.sum(u * b.bc_value * A)) * ENERGY_KCAL
                else:
                    sigma = -self.region_eps(self.outer(a)) * u
                    e["surface"] += -0.5 * float(np.sum(b.bc_value * sigma * A)) * ENERGY_KCAL
        e["total"] = e["coulomb"] + e["solvation"] + e["surface"]
        return e


def stern_sphere_solvation(q, a, b, eps_in, eps_out, kappa):
    """Closed form for a central charge q in a sphere of radius a (eps_in)
    inside an ion-free shell a < r < b (eps_out, no screening) in a solvent
    (eps_out, kappa), kcal/mol.  With phi = q/(4 pi eps_in r) + A (r < a),
    B/r + C (a < r < b), D e^{-kappa r}/r (r > b), continuity of phi and of
    eps dphi/dr at a and b give B = q/(4 pi eps_out), D e^{-kappa b} =
    B/(1 + kappa b), C = -B kappa/(1 + kappa b) and
    A = q/(4 pi) [1/(eps_out a) - kappa/(eps_out (1 + kappa b)) - 1/(eps_in a)];
    the solvation energy is q A / 2.  b = a is the screened Born sphere."""
    A = q / (4 * np.pi) * (1.0 / (eps_out * a) - kappa / (eps_out * (1 + kappa * b)) - 1.0 / (eps_in * a))
    return 0.5 * q * A * ENERGY_KCAL


def concentric_cavity_solvation(q, c, a, b, eps_cav, eps_mol, eps_out, kappa, lmax=60):
    """Solvation energy (kcal/mol) of a point charge q at distance c from the
    centre of a dielectric sphere of radius b (eps_mol) that holds a
    concentric spherical cavity of radius a < c (eps_cav, no screening), in a
    solvent (eps_out, kappa).  Legendre series: per degree l the potential is
    A r^l in the cavity, the charge's own term q/(4 pi eps_mol) r_<^l /
    r_>^(l+1) plus B r^l + C r^-(l+1) in the molecule, and D k_l(kappa r) in
    the solvent (k_l the modified spherical Bessel function of the second
    kind; r^-(l+1) when kappa = 0); continuity of phi and of eps dphi/dr at
    r = a and r = b fixes A, B, C, D, and phi_reac at the charge is
    sum_l (B c^l + C c^-(l+1)).  eps_cav = eps_mol removes the cavity."""
    from scipy.special import spherical_kn
    qm = q / (4 * np.pi * eps_mol)
    phi = 0.0
    for l in range(lmax + 1):
        if kappa > 0:
            kb, dkb = spherical_kn(l, kappa * b), kappa * spherical_kn(l, kappa * b, derivative=True)
        else:
            kb, dkb = b ** (-(l + 1)), -(l + 1) * b ** (-(l + 2))
        # unknowns (A, B, C, D)
        M = np.array([
            [a ** l, -a ** l, -a ** (-(l + 1)), 0.0],
            [eps_cav * l * a ** (l - 1) if l else 0.0, -eps_mol * l * a ** (l - 1) if l else 0.0,
             eps_mol * (l + 1) * a ** (-(l + 2)), 0.0],
            [0.0, b ** l, b ** (-(l + 1)), -kb],
            [0.0, eps_mol * l * b ** (l - 1) if l else 0.0, -eps_mol * (l + 1) * b ** (-(l + 2)), -eps_out * dkb],
        ])
        rhs = np.array([
            qm * a ** l / c ** (l + 1),
            eps_mol * qm * l * a ** (l - 1) / c ** (l + 1) if l else 0.0,
            -qm * c ** l / b ** (l + 1),
            eps_mol * qm * (l + 1) * c ** l / b ** (l + 2),
        ])
        A_, B_, C_, D_ = np.linalg.solve(M, rhs)
        phi += B_ * c ** l + C_ * c ** (-(l + 1))
    return 0.5 * q * phi * ENERGY_KCAL


class RegionTreecode:
    """Treecode product of a RegionSystem (the per-region rows above): per
    region R, the truncated expansion and near sums of oracle.treecode with
    R's screening, over the bodies bounding R with their signed side
    densities, plus R's tiered corrections; then row = jump - U_R.  Trees,
    target groups and interaction lists are those of oracle.treecode
    (Section 3.2 readings there); only the kernel and the densities depend on
    the region."""

    def __init__(self, rs, theta=None, P=None):
        from .treecode import BodyTree, interaction_lists
        self.rs = rs
        p = rs.p
        self.theta = p.theta if theta is None else theta
        self.P = p.P if P is None else P
        self.trees = [BodyTree(b, pn, p.K, p.leaf_size) for b, pn in zip(rs.bodies, rs.panels)]
        self.y, self.w = zip(*[pn.points(p.K) for pn in rs.panels])
        self.groups = []
        for a, (tr, pn) in enumerate(zip(self.trees, rs.panels)):
            for g0 in range(0, pn.N, p.group_size):
                idx = tr.perm[g0:g0 + p.group_size]
                x = pn.c[idx]
                self.groups.append((a, idx, x.min(0), x.max(0)))
        self.lists = {(gi, b): interaction_lists(tr, lo, hi, self.theta)
                      for gi, (a, idx, lo, hi) in enumerate(self.groups) for b, tr in enumerate(self.trees)}
        self.regions = sorted({R for b in range(len(rs.bodies)) for R in (rs.inner(b), rs.outer(b)) if R is not None})

    def _side(self, x, b, s, R):
        """(psi, phi) of body b seen from region R with the sign s folded in
        (unknowns only: the imposed values belong to the right-hand side)."""
        rs = self.rs
        bb = rs.bodies[b]
        N = rs.panels[b].N
        if bb.kind == DIELECTRIC:
            phi, dphi = rs.blocks(x, b)
            psi = dphi if s > 0 else (bb.eps_in / rs.region_eps(R)) * dphi
        elif bb.kind == SET_POTENTIAL:
            (psi,) = rs.blocks(x, b)
            phi = np.zeros(N)
        else:
            (phi,) = rs.blocks(x, b)
            psi = np.zeros(N)
        return s * psi, s * phi

    def _region_sum(self, x, R):
        from .integrals import kernel_terms
        from .treecode import _Sub, truncated_kernel
        rs = self.rs
        p = rs.p
        kap = rs.region_kappa(R)
        lap = kap == 0
        bnd = dict(rs.boundary(R))
        U = {a: np.zeros(rs.panels[a].N) for a in bnd}
        side = {b: self._side(x, b, s, R) for b, s in bnd.items()}
        pick = (lambda t: (t[0], t[1])) if lap else (lambda t: (t[2], t[3]))
        for gi, (a, idx, lo, hi) in enumerate(self.groups):
            if a not in bnd:
                continue
            xt = rs.panels[a].c[idx]
            for b in bnd:
                psi, phi = side[b]
                tr = self.trees[b]
                near, far = self.lists[(gi, b)]
                K = p.K
                q = self.w[b] * psi[:, None]
                pv = (self.w[b] * phi[:, None])[..., None] * rs.panels[b].n[:, None, :]
                for nid in near:
                    nd = tr.nodes[nid]
                    pj = tr.perm[nd["start"]:nd["end"]]
                    y = self.y[b][pj].reshape(-1, 3)
                    nrm = np.repeat(rs.panels[b].n[pj], K, axis=0)
                    g, k = pick(kernel_terms(xt[:, None, :], y[None], nrm[None], kap))
                    wphi = (pv[pj].reshape(-1, 3) * nrm).sum(-1)
                    U[a][idx] += g @ q[pj].reshape(-1) - k @ wphi
                for nid in far:
                    nd = tr.nodes[nid]
                    pj = tr.perm[nd["start"]:nd["end"]]
                    c = nd["center"]
                    y = self.y[b][pj].reshape(-1, 3)
                    Rv = (xt - c)[:, None, :] * np.ones((1, len(y), 1))
                    dvec = np.broadcast_to((y - c)[None], Rv.shape)
                    pp = np.broadcast_to(pv[pj].reshape(-1, 3)[None], Rv.shape)
                    F, dF = truncated_kernel(Rv, dvec, pp, kap, self.P, lap)
                    U[a][idx] += F @ q[pj].reshape(-1) - dF.sum(1)
        # tiered corrections among the region's bodies
        for a in bnd:
            pa = rs.panels[a]
            for b in bnd:
                pb = rs.panels[b]
                psi, phi = side[b]
                dc = pa.c[:, None, :] - pb.c[None, :, :]
                near = np.einsum("ijk,ijk->ij", dc, dc) < 8.0 * pb.A[None, :]
                if a == b:
                    near[np.arange(pa.N), np.arange(pa.N)] = True
                for i, j in zip(*np.nonzero(near)):
                    tier = pick(panel_operator_blocks(pa.c[i:i + 1], _Sub(pb, j), kap, p.K, p.K_near, p.n_edge,
                                                      np.array([0 if (a == b and i == j) else -1])))
                    kp = pick(kernel_terms(pa.c[i][None, :], self.y[b][j], pb.n[j][None, :], kap))
                    dV = tier[0][0, 0] - float((kp[0] * self.w[b][j]).sum())
                    dK = tier[1][0, 0] - float((kp[1] * self.w[b][j]).sum())
                    U[a][i] += dV * psi[j] - dK * phi[j]
        return U

    def apply(self, x):
        """A x of the per-region rows (same as RegionSystem.assemble()[0] @ x
        up to the treecode truncation)."""
        rs = self.rs
        out = np.zeros(rs.n)
        for a, ba in enumerate(rs.bodies):
            Na = rs.panels[a].N
            for r0, R in rs.rows(a):
                if ba.kind == DIELECTRIC or ba.kind == SET_CHARGE:
                    out[r0:r0 + Na] = 0.5 * x[rs.offsets[a]:rs.offsets[a] + Na]
        for R in self.regions:
            for a, Ua in self._region_sum(x, R).items():
                for r0, Ra in self.rs.rows(a):
                    if Ra == R:
                        out[r0:r0 + rs.panels[a].N] -= Ua
        return out

"""Flat-panel geometry (Section 3.1).

The boundaries are flat triangles with piecewise-constant unknowns, collocated
at the panel centroids.  Normals point out of each body into the solvent
(reading G4: with this orientation the printed jump terms +1/2 of Eq. 5 hold,
and the Laplace double layer of a closed surface sums to -1/2 per row).
All arithmetic is FP64; sums are evaluated left to right, ((a+b)+c).
"""
import numpy as np

from .quadrature import triangle_rule


def rigid_transform(verts, R=None, t=None):
    """World-frame vertices R v + t, each component evaluated as
    ((R0 v0 + R1 v1) + R2 v2) + t (left to right, no fused products)."""
    v = np.asarray(verts, dtype=np.float64)
    if R is None and t is None:
        return v.copy()
    R = np.eye(3) if R is None else np.asarray(R, dtype=np.float64)
    t = np.zeros(3) if t is None else np.asarray(t, dtype=np.float64)
    out = np.empty_like(v)
    for a in range(3):
        out[:, a] = ((R[a, 0] * v[:, 0] + R[a, 1] * v[:, 1]) + R[a, 2] * v[:, 2]) + t[a]
    return out


class Panels:
    """Geometry of one triangulated boundary: vertices v0,v1,v2 (N,3) each,
    centroid c, unit normal n (out of the body), area A and L = sqrt(2A)."""

    def __init__(self, verts, tris):
        verts = np.asarray(verts, dtype=np.float64)
        tris = np.asarray(tris, dtype=np.int64)
        self.v = verts[tris]                         # (N,3,3)
        v0, v1, v2 = self.v[:, 0], self.v[:, 1], self.v[:, 2]
        self.c = ((v0 + v1) + v2) / 3.0
        cr = np.cross(v1 - v0, v2 - v0)
        nrm = np.sqrt(np.einsum("ij,ij->i", cr, cr))
        if np.any(nrm <= 0) or not np.all(np.isfinite(nrm)):
            raise ValueError("degenerate panel")
        self.n = cr / nrm[:, None]
        self.A = 0.5 * nrm
        self.L = np.sqrt(2.0 * self.A)               # Section 3.1: L = sqrt(2 A_j)
        self.N = len(tris)

    def points(self, K: int):
        """Quadrature points and weights of the K-point rule on every panel:
        y = c + sum_a mu_a (v_a - c); weights w_m * A_j.  Shapes (N,K,3), (N,K)."""
        mu, w = triangle_rule(K)
        d = self.v - self.c[:, None, :]              # (N,3,3) vertex offsets
        y = self.c[:, None, :] + np.einsum("ma,nad->nmd", mu, d)
        return y, w[None, :] * self.A[:, None]

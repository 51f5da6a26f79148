"""Panel integrals of the Laplace and Yukawa single and double layers
(Eq. 3-4, Eq. 8-9 and the three-tier rule of Section 3.1).

  G_L(r) = 1/(4 pi r),  G_Y(r) = exp(-kappa r)/(4 pi r)   (Eq. 4; reading G13:
  the Yukawa kernel is radial in r = |x - y|).
  V_ij = int_panel_j G(x_i, y) dA_y,
  K_ij = int_panel_j dG/dn_y dA_y,  dG/dn_y = n_j . grad_y G(x - y)
       = n_j.(x - y) G'(r)-term:  Laplace n.(x-y)/(4 pi r^3),
                                   Yukawa  n.(x-y)(1+kappa r) e^{-kappa r}/(4 pi r^3).

Tiers (Section 3.1):
  * the panel holding the collocation point: semi-analytical (reading G6),
    K_ii = 0 for a flat panel (reading G5);
  * centroid distance |x_i - c_j| < 2 L_j (strict, reading G7): fine rule;
  * otherwise the K-point far rule.
In the K-point and fine sums a quadrature node at distance exactly zero from
the target contributes nothing (only the self panel's centroid node can).
"""
import math

import numpy as np

from .quadrature import gauss_legendre01

FOUR_PI = 4.0 * math.pi


def kernel_terms(x, y, n, kappa):
    """Pointwise kernels for targets x (...,3), sources y (...,3), source
    normals n (...,3).  Returns (G_L, dG_L/dn_y, G_Y, dG_Y/dn_y); zero where
    r == 0."""
    d = x - y
    r2 = np.einsum("...i,...i->...", d, d)
    ok = r2 > 0
    r = np.sqrt(np.where(ok, r2, 1.0))
    nd = np.einsum("...i,...i->...", n, d)
    gl = np.where(ok, 1.0 / (FOUR_PI * r), 0.0)
    kl = np.where(ok, nd / (FOUR_PI * r ** 3), 0.0)
    e = np.exp(-kappa * r)
    gy = np.where(ok, e / (FOUR_PI * r), 0.0)
    ky = np.where(ok, nd * (1.0 + kappa * r) * e / (FOUR_PI * r ** 3), 0.0)
    return gl, kl, gy, ky


def rule_integrals(x, y, w, n, kappa):
    """sum_m w_m * kernels(x, y_m) over the last point axis.
    x (T,3) targets, y (T,K,3) or (K,3) nodes, w matching weights, n normals."""
    gl, kl, gy, ky = kernel_terms(x[:, None, :], y, n[:, None, :] if n.ndim == 2 else n, kappa)
    return ((gl * w).sum(-1), (kl * w).sum(-1), (gy * w).sum(-1), (ky * w).sum(-1))


def self_integral(v, c, kappa, n_edge: int):
    """Semi-analytical single-layer integral of a flat panel over itself at its
    centroid c (reading G6 of Section 3.1, after Hess-Smith / Zhu et al.):
    split the panel at c into three sub-triangles; in polar coordinates about c
    the radial integral is analytic, int_0^rho G(r) r dr = F(rho) with
    F_L = rho/(4 pi) and F_Y = (1 - exp(-kappa rho))/(4 pi kappa), and the
    angular integral is taken along each edge, d(theta) = h ds / rho(s)^2, by an
    n_edge-point Gauss-Legendre rule.  Returns (V_L, V_Y); K_ii = 0.
    v: (3,3) vertices, c: (3,) centroid."""
    s01, w01 = gauss_legendre01(n_edge)
    VL = 0.0
    VY = 0.0
    for a in range(3):
        pa, pb = v[a], v[(a + 1) % 3]
        e = pb - pa
        ell = math.sqrt(float(e @ e))
        u = e / ell
        foot = pa + ((c - pa) @ u) * u
        h = math.sqrt(float((c - foot) @ (c - foot)))
        p = pa[None, :] + (s01 * ell)[:, None] * u[None, :]
        rho = np.sqrt(np.einsum("ij,ij->i", p - c, p - c))
        jac = h / rho ** 2 * ell * w01
        VL += float(np.sum(rho / FOUR_PI * jac))
        if kappa > 0:
            VY += float(np.sum((1.0 - np.exp(-kappa * rho)) / (FOUR_PI * kappa) * jac))
        else:
            VY += float(np.sum(rho / FOUR_PI * jac))
    return VL, VY


def panel_operator_blocks(targets, panels, kappa, K, K_near, n_edge, self_index=None,
                          laplace=True):
    """Dense blocks V_L, K_L, V_Y, K_Y (T x N) of the discrete operators of
    Eq. 9 for target points `targets` (T,3) and source `panels`, with the
    three-tier rule selection of Section 3.1.  self_index[t] = j when target t
    is the centroid of source panel j (self tier), else -1."""
    T = len(targets)
    N = panels.N
    y, w = panels.points(K)
    yn, wn = panels.points(K_near)
    out = [np.zeros((T, N)) for _ in range(4)]
    chunk = max(1, 2_000_000 // max(1, N * K))
    for t0 in range(0, T, chunk):
        t1 = min(T, t0 + chunk)
        x = targets[t0:t1]
        gl, kl, gy, ky = kernel_terms(x[:, None, None, :], y[None], panels.n[None, :, None, :], kappa)
        vals = [(g * w[None]).sum(-1) for g in (gl, kl, gy, ky)]
        for o, v in zip(out, vals):
            o[t0:t1] = v
    # fine tier: |x_t - c_j| < 2 L_j  <=>  |x_t - c_j|^2 < 8 A_j
    dc = targets[:, None, :] - panels.c[None, :, :]
    d2 = np.einsum("tjd,tjd->tj", dc, dc)
    near = d2 < 8.0 * panels.A[None, :]
    if self_index is not None:
        for t, j in enumerate(self_index):
            if j >= 0:
                near[t, j] = False
    ti, tj = np.nonzero(near)
    if len(ti):
        gl, kl, gy, ky = kernel_terms(targets[ti][:, None, :], yn[tj], panels.n[tj][:, None, :], kappa)
        for o, g in zip(out, (gl, kl, gy, ky)):
            o[ti, tj] = (g * wn[tj]).sum(-1)
    if self_index is not None:
        for t, j in enumerate(self_index):
            if j >= 0:
                VL, VY = self_integral(panels.v[j], panels.c[j], kappa, n_edge)
                out[0][t, j] = VL
                out[1][t, j] = 0.0
                out[2][t, j] = VY
                out[3][t, j] = 0.0
    return tuple(out)

"""Treecode approximation of the boundary-element matvec (Section 3.2).

The paper accelerates the matvec, an N-body sum with Gauss points as sources
and collocation points as targets, by a Barnes-Hut treecode with a Cartesian
Taylor expansion of order P and a multipole acceptance criterion theta; it
defers the details to earlier work.  The oracle's reading (G9, G21), stated so
that a second implementation reproduces the same interaction lists:

  Tree (one per body, built from body-frame panel centroids):
    * bounding cube: lo = min of the centroids per axis, ext = max extent
      (1 if zero); 10-bit cell index per axis q = floor((c - lo) * (1024/ext)),
      clamped to 1023; 30-bit Morton key with x in the highest bit of each
      triple; panels stably sorted by key (ties keep input order).
    * a node at depth l holds the panels sharing the top 3l key bits; it is
      split into its non-empty octants (in key order) while it holds more
      than leaf_size panels and l < 10.
    * node centre: the cube cell centre lo + h (2 i + 1), h = ext 2^-(l+1),
      mapped to the world frame; radius r_b: max distance from that centre to
      the K-point quadrature nodes of the node's panels (world frame).
  Target groups: per body, consecutive runs of group_size panels in key order;
    a group's box is the axis-aligned box of its world-frame centroids.
  Acceptance: a node is far for a group when theta > 0 and
    r_b^2 <= theta^2 d^2, d = distance from the node centre to the group box
    (ties count as far); otherwise a leaf is near and an inner node is opened.
    Lists are produced depth first, children in key order, bodies in order.
  Far nodes: every source point s of the node contributes the degree-<=P part
    of the Taylor expansion of its kernel about the node centre c_b.
  Near leaves: the K-point sum, nodes at distance zero skipped.
  Near-field corrections: for every target i and source panel j with
    |x_i - c_j| < 2 L_j, or j the panel of x_i, the tiered entry of
    Section 3.1 replaces the K-point entry: tiered minus K-point is added.

Truncated expansion, computed by univariate Taylor arithmetic: with
R = x - c_b and d = y - c_b, f(t) = G(|R - t d|) = sum_n c_n t^n, and the
degree-n homogeneous part of the Cartesian expansion in d is c_n, so the
truncated kernel is F_P(d) = sum_{n<=P} c_n.  The double layer needs
p . grad_d F_P(d); it is the epsilon-part of the same series taken over dual
numbers a + b*epsilon with d replaced by d + epsilon p.  The series of
rho^2(t) = |R|^2 - 2 t R.d + t^2 |d|^2 is exact; sqrt, reciprocal and exp of a
power series use the standard recurrences.
"""
import math

import numpy as np

from .bem import DIELECTRIC, SET_CHARGE, System
from .geometry import Panels, rigid_transform
from .integrals import kernel_terms, panel_operator_blocks

FOUR_PI = 4.0 * math.pi


def morton_keys(c_body):
    lo = c_body.min(axis=0)
    hi = c_body.max(axis=0)
    ext = float(np.max(hi - lo))
    if ext <= 0:
        ext = 1.0
    s = 1024.0 / ext
    q = np.floor((c_body - lo[None, :]) * s).astype(np.int64)
    q = np.clip(q, 0, 1023)
    key = np.zeros(len(c_body), dtype=np.int64)
    for b in range(10):
        key |= ((q[:, 0] >> b) & 1) << (3 * b + 2)
        key |= ((q[:, 1] >> b) & 1) << (3 * b + 1)
        key |= ((q[:, 2] >> b) & 1) << (3 * b)
    return key, q, lo, ext


class BodyTree:
    def __init__(self, body, panels, K, leaf_size):
        vb = np.asarray(body.verts, dtype=np.float64)[np.asarray(body.tris)]
        cb = ((vb[:, 0] + vb[:, 1]) + vb[:, 2]) / 3.0
        key, q, lo, ext = morton_keys(cb)
        self.perm = np.argsort(key, kind="stable")
        self.key = key[self.perm]
        self.q = q[self.perm]
        self.lo, self.ext = lo, ext
        self.nodes = []          # dicts: level, start, end, children, center
        self.leaf_size = leaf_size
        self._build(0, 0, len(key))
        y, w = panels.points(K)
        ys = y[self.perm]        # (N,K,3) in sorted order
        for nd in self.nodes:
            l = nd["level"]
            cell = self.q[nd["start"]] >> (10 - l)
            h = ext * 2.0 ** (-(l + 1))
            cbody = lo + h * (2 * cell + 1)
            cw = rigid_transform(cbody[None, :], body.R, body.t)[0]
            nd["center"] = cw
            d = ys[nd["start"]:nd["end"]].reshape(-1, 3) - cw[None, :]
            nd["r2"] = float(np.max((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]))

    def _build(self, level, start, end):
        idx = len(self.nodes)
        self.nodes.append({"level": level, "start": start, "end": end, "children": []})
        if end - start > self.leaf_size and level < 10:
            shift = 3 * (10 - (level + 1))
            oct_ = (self.key[start:end] >> shift) & 7
            for o in range(8):
                sel = np.nonzero(oct_ == o)[0]
                if len(sel):
                    ch = self._build(level + 1, start + int(sel[0]), start + int(sel[-1]) + 1)
                    self.nodes[idx]["children"].append(ch)
        return idx


def _mac_far(theta, r2, c, lo, hi):
    if theta <= 0:
        return False
    e = np.maximum(np.maximum(lo - c, c - hi), 0.0)
    d2 = (e[0] * e[0] + e[1] * e[1]) + e[2] * e[2]
    return r2 <= (theta * theta) * d2


def interaction_lists(tree, glo, ghi, theta):
    near, far = [], []
    stack = [0]
    while stack:
        i = stack.pop()
        nd = tree.nodes[i]
        if _mac_far(theta, nd["r2"], nd["center"], glo, ghi):
            far.append(i)
        elif not nd["children"]:
            near.append(i)
        else:
            stack.extend(reversed(nd["children"]))
    return near, far


# ---- dual-number power series -------------------------------------------
def _mul(a, b):
    return (a[0] * b[0], a[0] * b[1] + a[1] * b[0])


def _div(a, b):
    return (a[0] / b[0], (a[1] * b[0] - a[0] * b[1]) / (b[0] * b[0]))


def _add(a, b):
    return (a[0] + b[0], a[1] + b[1])


def truncated_kernel(R, d, p, kappa, P, laplace):
    """(F_P(d), p.grad_d F_P(d)) for G = 1/(4 pi rho) (laplace) or
    exp(-kappa rho)/(4 pi rho), rho = |R - d|; arrays over pairs (...,3)."""
    z = np.zeros(R.shape[:-1])
    RR = np.einsum("...i,...i->...", R, R)
    Rd = np.einsum("...i,...i->...", R, d)
    Rp = np.einsum("...i,...i->...", R, p)
    dd = np.einsum("...i,...i->...", d, d)
    dp = np.einsum("...i,...i->...", d, p)
    a = [(RR, z), (-2 * Rd, -2 * Rp), (dd, 2 * dp)] + [(z, z)] * (P - 2 if P > 2 else 0)
    a = a[:P + 1] if P >= 2 else a[:P + 1]
    while len(a) < P + 1:
        a.append((z, z))
    s0v = np.sqrt(RR)
    s = [(s0v, z)]
    two_s0 = (2 * s0v, z)
    for n in range(1, P + 1):
        acc = a[n]
        for k in range(1, n):
            m = _mul(s[k], s[n - k])
            acc = (acc[0] - m[0], acc[1] - m[1])
        s.append(_div(acc, two_s0))
    r = [_div((np.ones_like(z), z), s[0])]
    for n in range(1, P + 1):
        acc = (z, z)
        for k in range(1, n + 1):
            acc = _add(acc, _mul(s[k], r[n - k]))
        q = _div(acc, s[0])
        r.append((-q[0], -q[1]))
    if laplace:
        G = r
    else:
        g = [(-kappa * x[0], -kappa * x[1]) for x in s]
        e0 = np.exp(g[0][0])
        E = [(e0, e0 * g[0][1])]
        for n in range(1, P + 1):
            acc = (z, z)
            for k in range(1, n + 1):
                m = _mul(g[k], E[n - k])
                acc = (acc[0] + k * m[0], acc[1] + k * m[1])
            E.append((acc[0] / n, acc[1] / n))
        G = []
        for n in range(P + 1):
            acc = (z, z)
            for k in range(n + 1):
                acc = _add(acc, _mul(E[k], r[n - k]))
            G.append(acc)
    F = sum(x[0] for x in G) / FOUR_PI
    dF = sum(x[1] for x in G) / FOUR_PI
    return F, dF


class TreecodeOperator:
    """Treecode matvec of a System (same rows as System.apply).

    groups: optional indices of target groups (numbered over the bodies in
    order, group_size targets each in Morton order) to which the product is
    restricted; apply() then returns NaN in the rows of every other target.
    The lists, corrections and sums of the kept targets are unchanged."""

    def __init__(self, sys: System, theta=None, P=None, groups=None):
        self.sys = sys
        p = sys.p
        self.theta = p.theta if theta is None else theta
        self.P = p.P if P is None else P
        self.trees = [BodyTree(b, pn, p.K, p.leaf_size) for b, pn in zip(sys.bodies, sys.panels)]
        self.y, self.w = zip(*[pn.points(p.K) for pn in sys.panels])
        self.groups = []     # (body, target panel indices (original order), lo, hi)
        for a, (tr, pn) in enumerate(zip(self.trees, sys.panels)):
            for g0 in range(0, pn.N, p.group_size):
                idx = tr.perm[g0:g0 + p.group_size]
                x = pn.c[idx]
                self.groups.append((a, idx, x.min(0), x.max(0)))
        self.rows = None
        if groups is not None:
            self.groups = [self.groups[g] for g in groups]
            self.rows = [np.zeros(pn.N, dtype=bool) for pn in sys.panels]
            for a, idx, _, _ in self.groups:
                self.rows[a][idx] = True
        self.lists = {}
        for gi, (a, idx, lo, hi) in enumerate(self.groups):
            for b, tr in enumerate(self.trees):
                self.lists[(gi, b)] = interaction_lists(tr, lo, hi, self.theta)
        self._corrections()

    def _corrections(self):
        """Per target body a and source body b: sparse (i, j, dVL, dKL, dVY, dKY)."""
        sys = self.sys
        p = sys.p
        self.corr = {}
        for a, pa in enumerate(sys.panels):
            rows = np.arange(pa.N) if self.rows is None else np.nonzero(self.rows[a])[0]
            for b, pb in enumerate(sys.panels):
                dc = pa.c[rows][:, None, :] - pb.c[None, :, :]
                d2 = np.einsum("ijk,ijk->ij", dc, dc)
                near = d2 < 8.0 * pb.A[None, :]
                if a == b:
                    near[np.arange(len(rows)), rows] = True
                ii, jj = np.nonzero(near)
                ii = rows[ii]
                vals = np.zeros((len(ii), 4))
                for t, (i, j) in enumerate(zip(ii, jj)):
                    tier = panel_operator_blocks(pa.c[i:i + 1], _Sub(pb, j), sys.kappa, p.K, p.K_near,
                                                 p.n_edge, np.array([0 if (a == b and i == j) else -1]))
                    yk, wk = self.y[b][j], self.w[b][j]
                    kp = kernel_terms(pa.c[i][None, :], yk, pb.n[j][None, :], sys.kappa)
                    for m in range(4):
                        vals[t, m] = tier[m][0, 0] - float((kp[m] * wk).sum())
                self.corr[(a, b)] = (ii, jj, vals)

    def potentials(self, x):
        """U_L, U_Y per body (arrays over that body's panels, original order)."""
        sys = self.sys
        dens = [sys.densities(x, b) for b in range(len(sys.bodies))]
        srcs = []
        for b, pb in enumerate(sys.panels):
            psiL, phiL, psiY, phiY = dens[b]
            w = self.w[b]
            srcs.append(dict(y=self.y[b], qL=w * psiL[:, None], qY=w * psiY[:, None],
                             pL=(w * phiL[:, None])[..., None] * pb.n[:, None, :],
                             pY=(w * phiY[:, None])[..., None] * pb.n[:, None, :]))
        UL = [np.zeros(pn.N) for pn in sys.panels]
        UY = [np.zeros(pn.N) for pn in sys.panels]
        for gi, (a, idx, lo, hi) in enumerate(self.groups):
            xt = sys.panels[a].c[idx]
            for b, tr in enumerate(self.trees):
                lap = (a == b and sys.bodies[a].kind == DIELECTRIC)
                near, far = self.lists[(gi, b)]
                s = srcs[b]
                perm = tr.perm
                for nid in near:
                    nd = tr.nodes[nid]
                    pj = perm[nd["start"]:nd["end"]]
                    y = s["y"][pj].reshape(-1, 3)
                    nrm = np.repeat(sys.panels[b].n[pj], y.shape[0] // len(pj), axis=0)
                    gl, kl, gy, ky = kernel_terms(xt[:, None, :], y[None], nrm[None], sys.kappa)
                    # U = q G - p.grad_y G, with p = w phi n: n.grad_y G = kl/ky
                    wphiL = (s["pL"][pj].reshape(-1, 3) * nrm).sum(-1)
                    wphiY = (s["pY"][pj].reshape(-1, 3) * nrm).sum(-1)
                    if lap:
                        UL[a][idx] += gl @ s["qL"][pj].reshape(-1) - kl @ wphiL
                    UY[a][idx] += gy @ s["qY"][pj].reshape(-1) - ky @ wphiY
                for nid in far:
                    nd = tr.nodes[nid]
                    pj = perm[nd["start"]:nd["end"]]
                    c = nd["center"]
                    y = s["y"][pj].reshape(-1, 3)
                    R = (xt - c)[:, None, :] * np.ones((1, len(y), 1))
                    dvec = np.broadcast_to((y - c)[None], R.shape)
                    if lap:
                        pL = np.broadcast_to(s["pL"][pj].reshape(-1, 3)[None], R.shape)
                        F, dF = truncated_kernel(R, dvec, pL, 0.0, self.P, True)
                        UL[a][idx] += F @ s["qL"][pj].reshape(-1) - dF.sum(1)
                    pY = np.broadcast_to(s["pY"][pj].reshape(-1, 3)[None], R.shape)
                    F, dF = truncated_kernel(R, dvec, pY, sys.kappa, self.P, False)
                    UY[a][idx] += F @ s["qY"][pj].reshape(-1) - dF.sum(1)
        for (a, b), (ii, jj, vals) in self.corr.items():
            psiL, phiL, psiY, phiY = dens[b]
            if a == b and sys.bodies[a].kind == DIELECTRIC:
                np.add.at(UL[a], ii, vals[:, 0] * psiL[jj] - vals[:, 1] * phiL[jj])
            np.add.at(UY[a], ii, vals[:, 2] * psiY[jj] - vals[:, 3] * phiY[jj])
        return UL, UY

    def apply(self, x):
        sys = self.sys
        UL, UY = self.potentials(x)
        out = np.zeros(sys.n)
        for a, ba in enumerate(sys.bodies):
            o = sys.offsets[a]
            N = sys.panels[a].N
            if ba.kind == DIELECTRIC:
                phi, dphi = sys.blocks(x, a)
                out[o:o + N] = 0.5 * phi - UL[a]
                out[o + N:o + 2 * N] = 0.5 * phi + UY[a]
            else:
                (u,) = sys.blocks(x, a)
                out[o:o + N] = UY[a] + (0.5 * u if ba.kind == SET_CHARGE else 0.0)
        if self.rows is not None:
            for a, ba in enumerate(sys.bodies):
                o, N = sys.offsets[a], sys.panels[a].N
                for k in range(2 if ba.kind == DIELECTRIC else 1):
                    out[o + k * N:o + (k + 1) * N][~self.rows[a]] = np.nan
        return out


class _Sub:
    """One panel of a Panels object, as a Panels-like view."""

    def __init__(self, pn, j):
        self.v = pn.v[j:j + 1]
        self.c = pn.c[j:j + 1]
        self.n = pn.n[j:j + 1]
        self.A = pn.A[j:j + 1]
        self.L = pn.L[j:j + 1]
        self.N = 1
        self._pn, self._j = pn, j

    def points(self, K):
        # the rule of Panels.points applied to this one panel
        return Panels.points(self, K)

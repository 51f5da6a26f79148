"""Seeded synthetic inputs: triangle meshes, point charges and rigid poses.

This module generates the geometry and charges that both the CUDA path and the
CPU oracle consume.  It holds none of the boundary-element arithmetic (no
panel integrals, no operators, no energies): only vertex/triangle generation,
random coefficients and rejection sampling.

Conventions shared by every generator:
  * vertices are float64 arrays of shape (nv, 3) in Angstrom;
  * triangles are int32 arrays of shape (nt, 3), ordered counter-clockwise
    when seen from the solvent side, so that (v1-v0) x (v2-v0) points out of
    the body into the solvent (the normal convention of the paper's Eq. 2-3);
  * charges are (xyz (nq,3) float64 Angstrom, q (nq,) float64 in units of e).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "icosahedron", "icosphere", "geodesic_sphere", "star_radius", "star_surface",
    "star_coefficients", "interior_charges", "random_rotations", "translate",
    "rotate", "mesh_area", "nu_for_density", "brick",
]


def icosahedron():
    """Unit icosahedron: 12 vertices on the unit sphere, 20 outward-oriented faces."""
    p = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([
        [-1, p, 0], [1, p, 0], [-1, -p, 0], [1, -p, 0],
        [0, -1, p], [0, 1, p], [0, -1, -p], [0, 1, -p],
        [p, 0, -1], [p, 0, 1], [-p, 0, -1], [-p, 0, 1],
    ], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int32)
    return _orient_outward(v, f)


def _orient_outward(v, f):
    c = v[f].mean(axis=1)
    n = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = np.einsum("ij,ij->i", n, c) < 0
    f = f.copy()
    f[flip] = f[flip][:, [0, 2, 1]]
    return v, f


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Icosphere with 20*4**level faces: each subdivision splits a face into four
    at its edge midpoints, and every vertex is projected back onto the sphere."""
    v, f = icosahedron()
    verts = [tuple(x) for x in v]
    for _ in range(level):
        cache: dict = {}
        newf = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = np.add(verts[a], verts[b])
                m /= np.linalg.norm(m)
                cache[key] = len(verts)
                verts.append(tuple(m))
            return cache[key]

        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            newf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        f = np.array(newf, dtype=np.int32)
    v = np.array(verts, dtype=np.float64) * radius + np.asarray(center, dtype=np.float64)
    return v, f


def geodesic_sphere(nu: int):
    """Unit geodesic icosahedron of frequency nu: every icosahedron face is cut
    into nu*nu triangles on a barycentric grid, then projected onto the sphere.
    Returns (verts (nv,3), tris (20*nu*nu, 3))."""
    v0, f0 = icosahedron()
    index: dict = {}
    verts = []
    tris = []

    def vid(p):
        q = p / np.linalg.norm(p)
        key = tuple(np.round(q * 1e9).astype(np.int64))
        if key not in index:
            index[key] = len(verts)
            verts.append(q)
        return index[key]

    for a, b, c in f0:
        A, B, C = v0[a], v0[b], v0[c]
        ids = {}
        for i in range(nu + 1):
            for j in range(nu + 1 - i):
                k = nu - i - j
                ids[(i, j)] = vid((i * A + j * B + k * C) / nu)
        for i in range(nu):
            for j in range(nu - i):
                tris.append((ids[(i, j)], ids[(i + 1, j)], ids[(i, j + 1)]))
                if i + j + 1 < nu:
                    tris.append((ids[(i + 1, j)], ids[(i + 1, j + 1)], ids[(i, j + 1)]))
    v = np.array(verts, dtype=np.float64)
    f = np.array(tris, dtype=np.int32)
    return _orient_outward(v, f)


def _real_sph_harm(lmax, theta, phi):
    """Real orthonormal spherical harmonics Y_lm(theta, phi) for l <= lmax,
    as a dict (l, m) -> array.  theta is the polar angle."""
    x = np.cos(theta)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    # associated Legendre P_l^m without the Condon-Shortley phase
    P = {(0, 0): np.ones_like(x)}
    for m in range(1, lmax + 1):
        P[(m, m)] = P[(m - 1, m - 1)] * (2 * m - 1) * s
    for m in range(0, lmax):
        P[(m + 1, m)] = x * (2 * m + 1) * P[(m, m)]
    for m in range(0, lmax + 1):
        for l in range(m + 2, lmax + 1):
            P[(l, m)] = ((2 * l - 1) * x * P[(l - 1, m)] - (l + m - 1) * P[(l - 2, m)]) / (l - m)
    Y = {}
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
            if m == 0:
                Y[(l, m)] = norm * P[(l, 0)]
            elif m > 0:
                Y[(l, m)] = math.sqrt(2.0) * norm * P[(l, am)] * np.cos(am * phi)
            else:
                Y[(l, m)] = math.sqrt(2.0) * norm * P[(l, am)] * np.sin(am * phi)
    return Y


def star_coefficients(seed: int, lmax: int = 6, sigma: float = 0.03):
    """a_lm ~ N(0, sigma^2) for 0 <= l <= lmax, -l <= m <= l, drawn in (l, m) order."""
    rng = np.random.default_rng(seed)
    return {(l, m): float(rng.normal(0.0, sigma)) for l in range(lmax + 1) for m in range(-l, l + 1)}


def star_radius(dirs, coeffs, r0: float = 15.0):
    """r(theta, phi) = r0 * (1 + sum a_lm Y_lm(theta, phi)) along unit directions dirs (n,3)."""
    lmax = max(l for l, _ in coeffs)
    theta = np.arccos(np.clip(dirs[:, 2], -1.0, 1.0))
    phi = np.arctan2(dirs[:, 1], dirs[:, 0])
    Y = _real_sph_harm(lmax, theta, phi)
    f = np.ones(len(dirs))
    for key, a in coeffs.items():
        f = f + a * Y[key]
    return r0 * f


def mesh_area(verts, tris) -> float:
    e1 = verts[tris[:, 1]] - verts[tris[:, 0]]
    e2 = verts[tris[:, 2]] - verts[tris[:, 0]]
    return float(0.5 * np.linalg.norm(np.cross(e1, e2), axis=1).sum())


def nu_for_density(seed: int, density: float, r0: float = 15.0) -> int:
    """Geodesic frequency giving about `density` panels per square Angstrom:
    nu = round(sqrt(density * area / 20)), area measured on a nu=40 mesh."""
    v, f = star_surface(seed, 40, r0)
    return int(round(math.sqrt(density * mesh_area(v, f) / 20.0)))


def star_surface(seed: int, nu: int, r0: float = 15.0, lmax: int = 6, sigma: float = 0.03):
    """Star-shaped molecule: the geodesic sphere of frequency nu mapped radially
    to r(theta,phi) = r0 (1 + sum_{l<=lmax} a_lm Y_lm).  20*nu^2 panels."""
    u, f = geodesic_sphere(nu)
    r = star_radius(u, star_coefficients(seed, lmax, sigma), r0)
    v = u * r[:, None]
    return _orient_outward(v, f)


def interior_charges(seed: int, n: int, verts, tris, min_dist: float = 1.5,
                     qmax: float = 0.8, radius_fn=None):
    """n charges uniform inside a star-shaped closed mesh (rejection sampling):
    a point is kept when it is inside (radially below the surface) and at least
    `min_dist` from every vertex, edge midpoint and panel centroid.  Charges are
    q ~ U(-qmax, qmax) e."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    cen = verts[tris].mean(axis=1)
    mids = np.concatenate([(verts[tris[:, a]] + verts[tris[:, b]]) / 2 for a, b in ((0, 1), (1, 2), (2, 0))])
    kd = cKDTree(np.concatenate([verts, cen, mids]))
    # radial surface height along a direction: nearest-vertex radius is a
    # conservative stand-in only when radius_fn is absent
    vdir = verts / np.linalg.norm(verts, axis=1, keepdims=True)
    vkd = cKDTree(vdir)
    rmax = float(np.linalg.norm(verts, axis=1).max())
    out = []
    while len(out) < n:
        p = rng.uniform(-rmax, rmax, size=(4 * n, 3))
        rp = np.linalg.norm(p, axis=1)
        d = p / np.maximum(rp, 1e-300)[:, None]
        if radius_fn is not None:
            rs = radius_fn(d)
        else:
            _, idx = vkd.query(d, k=3)
            rs = np.linalg.norm(verts[idx], axis=2).min(axis=1)
        ok = rp < rs - min_dist
        dist, _ = kd.query(p)
        ok &= dist >= min_dist
        out.extend(p[ok].tolist())
    xyz = np.array(out[:n], dtype=np.float64)
    q = rng.uniform(-qmax, qmax, size=n)
    return xyz, q


def random_rotations(seed: int, n: int):
    """n uniform random rotation matrices from unit quaternions drawn with
    Shoemake's method (three uniforms per quaternion)."""
    rng = np.random.default_rng(seed)
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a = np.sqrt(1 - u1)
    b = np.sqrt(u1)
    w = a * np.sin(2 * np.pi * u2)
    x = a * np.cos(2 * np.pi * u2)
    y = b * np.sin(2 * np.pi * u3)
    z = b * np.cos(2 * np.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def rotate(xyz, R):
    return np.asarray(xyz) @ np.asarray(R).T


def translate(xyz, t):
    return np.asarray(xyz) + np.asarray(t, dtype=np.float64)


def brick(lx: float, ly: float, lz: float, h: float, center=(0.0, 0.0, 0.0)):
    """Closed surface of an axis-aligned box lx x ly x lz (Angstrom) centred at
    `center`: each face cut into squares of side close to h (at least one per
    edge), each square into two triangles; faces share their edge vertices
    (watertight) and every triangle is counter-clockwise seen from outside."""
    L = np.array([lx, ly, lz], dtype=float)
    n = np.maximum(1, np.round(L / h).astype(int))
    index = {}
    verts = []

    def vid(ijk):
        key = tuple(int(c) for c in ijk)
        if key not in index:
            index[key] = len(verts)
            verts.append([key[a] / n[a] * L[a] - 0.5 * L[a] for a in range(3)])
        return index[key]

    tris = []
    for axis in range(3):
        u, w = (axis + 1) % 3, (axis + 2) % 3          # (u, w, axis) is right-handed
        for side in (0, 1):
            for a in range(n[u]):
                for b in range(n[w]):
                    corner = []
                    for du, dw in ((0, 0), (1, 0), (1, 1), (0, 1)):
                        g = [0, 0, 0]
                        g[axis] = side * n[axis]
                        g[u] = a + du
                        g[w] = b + dw
                        corner.append(vid(g))
                    q = [corner[0], corner[1], corner[2], corner[3]]
                    if side == 0:                      # outward normal is -axis: reverse
                        q = q[::-1]
                    tris.append([q[0], q[1], q[2]])
                    tris.append([q[0], q[2], q[3]])
    v = np.asarray(verts, dtype=np.float64) + np.asarray(center, dtype=np.float64)
    return v, np.asarray(tris, dtype=np.int32)

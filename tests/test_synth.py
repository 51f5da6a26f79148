"""Synthetic meshes: the box surface used for the flat-faced charged body
(closed, outward-oriented, exact area and volume), and the oracle's
double-layer identity on it."""
from collections import Counter

import numpy as np

import synth


def _check_closed_outward(v, f):
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    edges = Counter()
    for t in f:
        for k in range(3):
            edges[(int(t[k]), int(t[(k + 1) % 3]))] += 1
    # every directed edge once, and its reverse once: closed and consistently oriented
    assert max(edges.values()) == 1
    assert all(edges[(j, i)] == 1 for (i, j) in edges)
    area = 0.5 * np.linalg.norm(np.cross(b - a, c - a), axis=1).sum()
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    return area, vol


def test_brick_is_closed_outward_with_exact_area_and_volume():
    for dims, h in (((100.0, 100.0, 10.0), 5.0), ((3.0, 2.0, 1.0), 0.7), ((1.0, 1.0, 1.0), 5.0)):
        v, f = synth.brick(*dims, h, center=(1.0, -2.0, 0.5))
        area, vol = _check_closed_outward(v - np.array([1.0, -2.0, 0.5]), f)
        lx, ly, lz = dims
        assert abs(area - 2 * (lx * ly + ly * lz + lx * lz)) < 1e-9 * area
        assert abs(vol - lx * ly * lz) < 1e-9 * vol
        assert np.allclose(v.min(0), np.array([1.0, -2.0, 0.5]) - 0.5 * np.array(dims))


def test_double_layer_of_a_brick_sums_to_minus_half():
    """Sum_j K_L,ij = -1/2 at every face centroid of a closed polyhedron (the
    solid angle of the surface seen from a point on a flat face is 2 pi),
    up to the quadrature error of the near panels."""
    from oracle.bem import SET_CHARGE, Body, Params, System
    v, f = synth.brick(4.0, 3.0, 2.0, 0.5)
    s = System([Body(SET_CHARGE, v, f, bc_value=0.0)], 80.0, 0.0, Params())
    VL, KL = s.operator_blocks(0, 0, True)[:2]
    rows = KL.sum(axis=1)
    assert np.abs(rows + 0.5).max() < 2e-3      # worst: next to an edge (measured 4.8e-4)
    assert np.median(np.abs(rows + 0.5)) < 1e-5  # away from edges the rules are near exact

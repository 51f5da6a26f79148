"""Direct pins of the oracle's octree and interaction lists (Section 3.2:
octree with N_crit panels per leaf, acceptance criterion theta, order P).

The CUDA lists are compared bit for bit with oracle/treecode.py, so these
tests check the oracle's tree and lists against their definitions by brute
force, independently of how treecode.py builds them:
  * every node is a cube of the body frame (its level fixes the edge) that
    contains the centroids of exactly its panels, its children split it and
    leaves hold at most N_crit panels;
  * r_b is the largest distance from the node centre to a K-point node of
    its panels;
  * every far (group, node) pair meets the criterion r_b <= theta |x - c_b|
    for every target x of the group, and no ancestor of a listed node did
    (the traversal opened it);
  * each group's near leaves and far nodes cover every source panel once;
  * with kappa = 0 and single-layer densities the treecode error of every
    row stays below the Legendre remainder bound
    sum_far |q_s| t^(P+1) / ((1 - t) 4 pi |x - c_b|), t = |y_s - c_b|/|x - c_b|,
    for P = 2..8.
"""
import math

import numpy as np
import pytest

import synth
from oracle.bem import DIELECTRIC, SET_POTENTIAL, Body, Params, System
from oracle.treecode import BodyTree, TreecodeOperator, interaction_lists

THETA = 0.5


def _system(leaf=16, kappa=0.125):
    """A posed star-shaped molecule (2000 panels) and a sphere (1280 panels)."""
    v, f = synth.star_surface(5, 10, 8.0)
    R = synth.random_rotations(17, 1)[0]
    mol = Body(DIELECTRIC, v, f, eps_in=4.0, charge_xyz=np.zeros((1, 3)), charge_q=np.array([1.0]),
               R=R, t=np.array([0.7, -1.1, 0.4]))
    v2, f2 = synth.icosphere(3, 4.0)
    srf = Body(SET_POTENTIAL, v2, f2, bc_value=1e-3, R=np.eye(3), t=np.array([15.5, 2.0, -1.0]))
    return System([mol, srf], 80.0, kappa, Params(leaf_size=leaf, group_size=32, theta=THETA))


@pytest.fixture(scope="module")
def trees():
    s = _system()
    return s, [BodyTree(b, pn, s.p.K, s.p.leaf_size) for b, pn in zip(s.bodies, s.panels)]


def _body_frame_centroids(body):
    v = np.asarray(body.verts, dtype=np.float64)[np.asarray(body.tris)]
    return v.mean(axis=1)


def _to_body(body, xw):
    R = np.eye(3) if body.R is None else np.asarray(body.R)
    t = np.zeros(3) if body.t is None else np.asarray(body.t)
    return (np.asarray(xw) - t) @ R   # R^T (x - t), row vectors


def _ancestors(tree):
    par = {}
    for i, nd in enumerate(tree.nodes):
        for ch in nd["children"]:
            par[ch] = i
    return par


def test_nodes_are_cubes_holding_exactly_their_panels(trees):
    s, trs = trees
    for body, tr in zip(s.bodies, trs):
        cb = _body_frame_centroids(body)
        ext = float(np.max(cb.max(0) - cb.min(0)))
        seen = {}
        for i, nd in enumerate(tr.nodes):
            h = ext * 2.0 ** -(nd["level"] + 1)          # half edge at this level
            cc = _to_body(body, nd["center"][None, :])[0]
            mine = tr.perm[nd["start"]:nd["end"]]
            slack = 1e-9 * ext
            # the node's panels lie in its cube ...
            assert np.all(np.abs(cb[mine] - cc[None, :]) <= h + slack)
            # ... and no other panel lies strictly inside it
            inside = np.all(np.abs(cb - cc[None, :]) < h - slack, axis=1)
            others = np.setdiff1d(np.nonzero(inside)[0], mine)
            assert len(others) == 0
            # one node per cube and level
            key = (nd["level"], tuple(np.round(cc / h).astype(np.int64)))
            assert key not in seen
            seen[key] = i
            if nd["children"]:
                assert nd["end"] - nd["start"] > s.p.leaf_size
                kids = [tr.nodes[c] for c in nd["children"]]
                assert kids[0]["start"] == nd["start"] and kids[-1]["end"] == nd["end"]
                for a, b in zip(kids[:-1], kids[1:]):
                    assert a["end"] == b["start"]
                for k in kids:
                    assert k["level"] == nd["level"] + 1
                    kc = _to_body(body, k["center"][None, :])[0]
                    # a child's cube is one octant of its parent's
                    np.testing.assert_allclose(np.abs(kc - cc), h / 2, rtol=0, atol=slack)
            else:
                assert nd["end"] - nd["start"] <= s.p.leaf_size or nd["level"] == 10
        # the root holds every panel
        assert tr.nodes[0]["start"] == 0 and tr.nodes[0]["end"] == len(cb)
        assert sorted(tr.perm.tolist()) == list(range(len(cb)))


def test_node_radius_is_the_farthest_quadrature_node(trees):
    s, trs = trees
    for b, tr in enumerate(trs):
        y, _ = s.panels[b].points(s.p.K)    # world frame, (N, K, 3)
        for nd in tr.nodes:
            pts = y[tr.perm[nd["start"]:nd["end"]]].reshape(-1, 3)
            d = np.sqrt(((pts - nd["center"][None, :]) ** 2).sum(1))
            assert math.sqrt(nd["r2"]) == pytest.approx(d.max(), rel=1e-13)
            # centroids alone would give a smaller radius on leaves of a few panels
        leaves = [nd for nd in tr.nodes if not nd["children"]]
        cen = s.panels[b].c
        gap = [math.sqrt(nd["r2"]) - np.sqrt(((cen[tr.perm[nd["start"]:nd["end"]]] - nd["center"]) ** 2).sum(1)).max()
               for nd in leaves]
        assert max(gap) > 0


def _groups(s, trs):
    out = []
    for a, (tr, pn) in enumerate(zip(trs, s.panels)):
        for g0 in range(0, pn.N, s.p.group_size):
            idx = tr.perm[g0:g0 + s.p.group_size]
            x = pn.c[idx]
            out.append((a, idx, x.min(0), x.max(0)))
    return out


def test_far_pairs_meet_the_criterion_for_every_target(trees):
    s, trs = trees
    n_far = 0
    for a, idx, lo, hi in _groups(s, trs):
        x = s.panels[a].c[idx]
        for tr in trs:
            near, far = interaction_lists(tr, lo, hi, THETA)
            par = _ancestors(tr)
            for nid in far:
                nd = tr.nodes[nid]
                dist = np.sqrt(((x - nd["center"]) ** 2).sum(1))
                assert np.all(math.sqrt(nd["r2"]) <= THETA * dist * (1 + 1e-14))
                n_far += 1
            for nid in list(far) + list(near):
                # every ancestor was opened: it failed the group criterion
                p = par.get(nid)
                while p is not None:
                    pn_ = tr.nodes[p]
                    e = np.maximum(np.maximum(lo - pn_["center"], pn_["center"] - hi), 0.0)
                    assert not (pn_["r2"] <= THETA ** 2 * float(e @ e))
                    p = par.get(p)
            for nid in near:
                assert not tr.nodes[nid]["children"]
    assert n_far > 0


def test_lists_cover_every_source_panel_once(trees):
    s, trs = trees
    for a, idx, lo, hi in _groups(s, trs):
        for b, tr in enumerate(trs):
            near, far = interaction_lists(tr, lo, hi, THETA)
            hit = np.zeros(s.panels[b].N, dtype=np.int64)
            for nid in list(near) + list(far):
                nd = tr.nodes[nid]
                hit[tr.perm[nd["start"]:nd["end"]]] += 1
            assert np.all(hit == 1)
        # theta = 0: everything is near (the direct sum)
        near0, far0 = interaction_lists(trs[0], lo, hi, 0.0)
        assert not far0 and sum(trs[0].nodes[i]["end"] - trs[0].nodes[i]["start"] for i in near0) == s.panels[0].N


@pytest.fixture(scope="module")
def laplace_operator():
    """kappa = 0 (both kernels Laplace), icospheres of 320 panels each."""
    v, f = synth.icosphere(2, 4.0)
    mol = Body(DIELECTRIC, v, f, eps_in=4.0, charge_xyz=np.zeros((1, 3)), charge_q=np.array([1.0]),
               R=synth.random_rotations(3, 1)[0], t=np.array([0.2, 0.1, -0.3]))
    v2, f2 = synth.icosphere(2, 3.0)
    srf = Body(SET_POTENTIAL, v2, f2, bc_value=1e-3, t=np.array([9.0, 1.0, 0.0]))
    s = System([mol, srf], 80.0, 0.0, Params(leaf_size=8, group_size=32, theta=THETA))
    return s, TreecodeOperator(s, theta=THETA, P=2)


@pytest.mark.parametrize("P", [2, 3, 4, 6, 8])
def test_single_layer_error_within_legendre_bound(laplace_operator, P):
    s, tc = laplace_operator
    tc.P = P   # the lists and near-field entries do not depend on P
    rng = np.random.default_rng(40 + P)
    x = np.zeros(s.n)
    N1 = s.panels[0].N
    x[N1:2 * N1] = rng.normal(size=N1)          # dphi/dn of the molecule (phi = 0)
    x[2 * N1:] = rng.normal(size=s.panels[1].N)  # dphi/dn of the held-potential surface
    err = tc.apply(x) - s.apply(x)
    # per row block: interior rows carry U_L (molecule sources only), exterior
    # and surface rows U_Y over both bodies; q_s = w_s psi_j
    dens = [s.densities(x, b) for b in range(2)]
    bound = np.zeros(s.n)
    for gi, (a, idx, lo, hi) in enumerate(tc.groups):
        xt = s.panels[a].c[idx]
        for b, tr in enumerate(tc.trees):
            _, far = tc.lists[(gi, b)]
            psiL, _, psiY, _ = dens[b]
            for nid in far:
                nd = tr.nodes[nid]
                pj = tr.perm[nd["start"]:nd["end"]]
                y = tc.y[b][pj].reshape(-1, 3)
                w = tc.w[b][pj]
                R = np.sqrt(((xt - nd["center"]) ** 2).sum(-1))     # (targets,)
                t = np.sqrt(((y - nd["center"]) ** 2).sum(-1))[None, :] / R[:, None]
                assert t.max() <= THETA * (1 + 1e-12)
                rem = t ** (P + 1) / ((1 - t) * 4 * math.pi * R[:, None])
                o = s.offsets[a]
                if a == b == 0:
                    bound[o + idx] += rem @ np.abs(w * psiL[pj, None]).reshape(-1)
                row = (o + N1 + idx) if a == 0 else (o + idx)
                bound[row] += rem @ np.abs(w * psiY[pj, None]).reshape(-1)
    tiny = 1e-13 * np.abs(s.apply(x)).max()
    assert np.all(np.abs(err) <= bound + tiny)
    # the bound is not vacuous: the error is a visible share of it somewhere
    assert np.max(np.abs(err) / (bound + tiny)) > 1e-3

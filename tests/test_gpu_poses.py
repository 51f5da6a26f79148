"""Rigid poses and the batched pose sweep (pgb_set_pose, pgb_solve_batch)
against the oracle and against physical invariances."""
import numpy as np
import pytest

import synth
from oracle.energy import energies
from oracle.treecode import TreecodeOperator
from problems import gpu_context, oracle_system, spheres, star_molecule

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_1506_03745_gb300 as pgb  # noqa: E402


def _posed_pair():
    mol = star_molecule(seed=5, nu=5, nq=20, r0=6.0)[0]
    v, f = synth.icosphere(2, 5.0)
    srf = dict(kind="sigma", verts=v, tris=f, eps_in=1.0, qxyz=np.zeros((0, 3)), q=np.zeros(0), bc=-0.05)
    return [mol, srf]


def _solve_energy(ctx, mode=None, tol=1e-10):
    n = pgb.pgb_num_unknowns(ctx)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    code, st = pgb.pgb_solve(ctx, pgb.PGB_FP64 if mode is None else mode, tol, 2000, 100, x)
    assert code == 0
    return x, pgb.pgb_energy(ctx, x)


def test_posed_geometry_matches_oracle():
    bodies = _posed_pair()
    R = synth.random_rotations(11, 1)[0]
    bodies[0]["R"], bodies[0]["t"] = R, np.array([0.5, -0.3, 0.2])
    bodies[1]["R"], bodies[1]["t"] = np.eye(3), np.array([14.0, 0.0, 0.0])
    so = oracle_system(bodies, theta=0.0)
    ctx = gpu_context(bodies, theta=0.0)
    try:
        _, e = _solve_energy(ctx)
        eo = energies(so, so.solve())
        for k in ("coulomb", "solvation", "surface", "total"):
            assert e[k] == pytest.approx(eo[k], rel=1e-8, abs=1e-12)
    finally:
        pgb.pgb_destroy(ctx)


def test_posed_treecode_lists_are_bit_exact():
    bodies = _posed_pair()
    R = synth.random_rotations(12, 1)[0]
    bodies[0]["R"], bodies[0]["t"] = R, np.array([0.0, 0.0, 0.0])
    bodies[1]["R"], bodies[1]["t"] = R.T, np.array([13.0, 1.0, -2.0])
    so = oracle_system(bodies, theta=0.5, P=4, leaf_size=8)
    ctx = gpu_context(bodies, theta=0.5, P=4, leaf_size=8)
    try:
        tc = TreecodeOperator(so)
        perm, noff, near, foff, far = pgb.pgb_tree_export(ctx)
        assert sum(len(tc.lists[k][1]) for k in tc.lists) == len(far)
        assert sum(len(tc.lists[k][0]) for k in tc.lists) == len(near)
        x = np.random.default_rng(4).normal(size=so.n)
        ref = tc.apply(x)
        xt = torch.tensor(x, device="cuda")
        yt = torch.empty_like(xt)
        pgb.pgb_matvec(ctx, xt, yt, pgb.PGB_FP64)
        assert np.abs(yt.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-10
    finally:
        pgb.pgb_destroy(ctx)


def test_common_rigid_motion_leaves_energies_unchanged():
    bodies = _posed_pair()
    bodies[1]["t"] = np.array([15.0, 0.0, 0.0])
    bodies[1]["R"] = np.eye(3)
    ctx = gpu_context(bodies, theta=0.0)
    try:
        _, e0 = _solve_energy(ctx)
        Q = synth.random_rotations(3, 1)[0]
        s = np.array([3.0, -7.0, 2.0])
        pgb.pgb_set_pose(ctx, 0, Q, s)
        pgb.pgb_set_pose(ctx, 1, Q, Q @ np.array([15.0, 0.0, 0.0]) + s)
        pgb.pgb_tree_build(ctx)
        _, e1 = _solve_energy(ctx)
        for k in ("solvation", "surface", "total"):
            assert e1[k] == pytest.approx(e0[k], rel=1e-9)
    finally:
        pgb.pgb_destroy(ctx)


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_batch_matches_one_pose_at_a_time(mode):
    bodies = _posed_pair()
    bodies[1]["t"] = np.array([15.0, 0.0, 0.0])
    bodies[1]["R"] = np.eye(3)
    Rs = synth.random_rotations(21, 3)
    ts = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [-1.0, 0.0, 1.0]])
    m = pgb.PGB_FP64 if mode == "fp64" else pgb.PGB_FP32
    ctx = gpu_context(bodies, theta=0.5, P=5, leaf_size=16)
    try:
        code, F, st = pgb.pgb_solve_batch(ctx, 0, Rs, ts, m, 1e-9 if mode == "fp64" else 1e-6, 2000, 100)
        assert code == 0 and len(st) == 3
        for b in range(3):
            c2 = gpu_context(bodies, theta=0.5, P=5, leaf_size=16)
            try:
                pgb.pgb_set_pose(c2, 0, Rs[b], ts[b])
                pgb.pgb_tree_build(c2)
                _, e = _solve_energy(c2, m, 1e-9 if mode == "fp64" else 1e-6)
            finally:
                pgb.pgb_destroy(c2)
            tol = 1e-8 if mode == "fp64" else 1e-5
            assert F[b, 3] == pytest.approx(e["total"], rel=tol)
            assert F[b, 1] == pytest.approx(e["solvation"], rel=tol)
        # poses differ, so the energies do
        assert np.ptp(F[:, 1]) > 0
    finally:
        pgb.pgb_destroy(ctx)


def test_fp32_mode_energy_error_against_fp64():
    bodies = spheres(kind="sigma", level_mol=3, level_srf=3)
    ctx = gpu_context(bodies, theta=0.5, P=6)
    try:
        _, e64 = _solve_energy(ctx, pgb.PGB_FP64, 1e-9)
        _, e32 = _solve_energy(ctx, pgb.PGB_FP32, 1e-6)
        _, er = _solve_energy(ctx, pgb.PGB_FP32_REFINE, 1e-6)
        for k in ("solvation", "surface", "total"):
            assert e32[k] == pytest.approx(e64[k], rel=1e-5)
            assert er[k] == pytest.approx(e64[k], rel=1e-5)
    finally:
        pgb.pgb_destroy(ctx)


def test_lanes_match_the_serial_batch():
    """Poses solved in concurrent lanes (own stream and host thread each)
    give the serial batch's energies, across calls that reuse the lanes, a
    change of charges and a move of the other body."""
    bodies = _posed_pair()
    bodies[1]["t"] = np.array([15.0, 0.0, 0.0])
    bodies[1]["R"] = np.eye(3)
    Rs = synth.random_rotations(31, 7)
    ts = np.stack([np.array([0.3 * k, -0.2 * k, 0.1]) for k in range(7)])
    c1 = gpu_context(bodies, theta=0.5, P=5, leaf_size=16, lanes=1)
    cl = gpu_context(bodies, theta=0.5, P=5, leaf_size=16, lanes=3)
    try:
        for step in range(3):
            if step == 1:  # new charges: the lanes are copied again
                q = bodies[0]["q"] * 0.7
                for c in (c1, cl):
                    pgb.pgb_set_charges(c, 0, q)
            if step == 2:  # the other body moves: the lanes follow
                for c in (c1, cl):
                    pgb.pgb_set_pose(c, 1, np.eye(3), [16.0, 1.0, 0.0])
            code1, F1, st1 = pgb.pgb_solve_batch(c1, 0, Rs, ts, pgb.PGB_FP64, 1e-9, 2000, 100)
            codel, Fl, stl = pgb.pgb_solve_batch(cl, 0, Rs, ts, pgb.PGB_FP64, 1e-9, 2000, 100)
            assert code1 == 0 and codel == 0
            np.testing.assert_allclose(Fl, F1, rtol=1e-12, atol=1e-14)
            assert [s["iterations"] for s in stl] == [s["iterations"] for s in st1]
            # both leave the body at the last pose with its tree built
            assert pgb.pgb_tree_stats(cl)["n_panels"] == pgb.pgb_tree_stats(c1)["n_panels"]
            _, e1 = _solve_energy(c1)
            _, el = _solve_energy(cl)
            assert el["total"] == pytest.approx(e1["total"], rel=1e-12)
            assert el["total"] == pytest.approx(F1[-1, 3], rel=1e-8)
    finally:
        pgb.pgb_destroy(c1)
        pgb.pgb_destroy(cl)

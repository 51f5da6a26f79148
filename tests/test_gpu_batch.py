"""Pose batches solved as one block-diagonal system (pgb_params.batch > 1,
pgb_solve_batch and pgb_solve_poses): every pose must come out as it does
when solved alone, across chunks, padding, several molecules of different
sizes and every solve mode."""
import numpy as np
import pytest

import synth
from problems import gpu_context, star_molecule

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_1506_03745_gb300 as pgb  # noqa: E402

TC = dict(theta=0.5, P=5, leaf_size=16)


def _surface():
    v, f = synth.icosphere(2, 5.0)
    return dict(kind="sigma", verts=v, tris=f, eps_in=1.0, qxyz=np.zeros((0, 3)), q=np.zeros(0), bc=-0.05,
                R=np.eye(3), t=np.array([15.0, 0.0, 0.0]))


def _pair(seed=5, nu=5, nq=20):
    return [star_molecule(seed=seed, nu=nu, nq=nq, r0=6.0)[0], _surface()]


def _poses(seed, B):
    Rs = synth.random_rotations(seed, B)
    ts = np.stack([np.array([0.2 * k, -0.15 * k, 0.1 * (k % 3)]) for k in range(B)])
    return Rs, ts


MODES = {"fp64": (pgb.PGB_FP64, 1e-9, 1e-9), "fp32": (pgb.PGB_FP32, 1e-6, 2e-6),
         "refine": (pgb.PGB_FP32_REFINE, 1e-8, 1e-8)}


@pytest.mark.parametrize("mode", sorted(MODES))
def test_union_batch_matches_serial_poses(mode):
    """7 poses in chunks of 3 (the last one padded) give the energies of the
    pose-by-pose batch, pose by pose, with the same iteration counts."""
    m, tol, rel = MODES[mode]
    Rs, ts = _poses(41, 7)
    # the serial reference without the overlapped FP64 residual, which the
    # batch does not use (both reach the same tolerance either way)
    c1 = gpu_context(_pair(), lanes=1, overlap=0, **TC)
    cb = gpu_context(_pair(), batch=3, **TC)
    try:
        code1, F1, st1 = pgb.pgb_solve_batch(c1, 0, Rs, ts, m, tol, 2000, 100)
        codeb, Fb, stb = pgb.pgb_solve_batch(cb, 0, Rs, ts, m, tol, 2000, 100)
        assert code1 == 0 and codeb == 0
        np.testing.assert_allclose(Fb, F1, rtol=rel, atol=1e-12)
        it1 = np.array([s["iterations"] for s in st1])
        itb = np.array([s["iterations"] for s in stb])
        assert np.abs(itb - it1).max() <= 1
        assert all(s["rel_residual"] <= tol for s in stb)
        assert np.ptp(Fb[:, 1]) > 0
        # a second call reuses the union (same chunk composition)
        code2, F2, _ = pgb.pgb_solve_batch(cb, 0, Rs, ts, m, tol, 2000, 100)
        assert code2 == 0
        np.testing.assert_allclose(F2, Fb, rtol=1e-12, atol=1e-14)
        # the body is left at the last pose with its tree built
        n = pgb.pgb_num_unknowns(cb)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        assert pgb.pgb_solve(cb, pgb.PGB_FP64, 1e-10, 2000, 100, x)[0] == 0
        assert pgb.pgb_energy(cb, x)["total"] == pytest.approx(F1[-1, 3], rel=max(rel, 1e-8))
    finally:
        pgb.pgb_destroy(c1)
        pgb.pgb_destroy(cb)


def test_union_batch_with_preconditioner():
    Rs, ts = _poses(43, 4)
    c1 = gpu_context(_pair(), lanes=1, precond=1, **TC)
    cb = gpu_context(_pair(), batch=4, precond=1, **TC)
    try:
        code1, F1, st1 = pgb.pgb_solve_batch(c1, 0, Rs, ts, pgb.PGB_FP64, 1e-9, 2000, 100)
        codeb, Fb, stb = pgb.pgb_solve_batch(cb, 0, Rs, ts, pgb.PGB_FP64, 1e-9, 2000, 100)
        assert code1 == 0 and codeb == 0
        np.testing.assert_allclose(Fb, F1, rtol=1e-9, atol=1e-12)
        assert [s["iterations"] for s in stb] == [s["iterations"] for s in st1]
    finally:
        pgb.pgb_destroy(c1)
        pgb.pgb_destroy(cb)


def test_solve_poses_molecules_of_different_sizes():
    """Two molecules (different meshes, charges and panel counts) near the
    same surface, interleaved in chunks of 4: each pose equals its molecule's
    own serial batch."""
    ca = gpu_context(_pair(seed=5, nu=5, nq=20), batch=4, **TC)
    cb = gpu_context(_pair(seed=9, nu=7, nq=35), **TC)
    refs = []
    try:
        na = pgb.pgb_tree_stats(ca)["n_panels"]
        nb = pgb.pgb_tree_stats(cb)["n_panels"]
        assert na != nb
        Rs, ts = _poses(47, 10)
        pose_ctx = np.array([k % 2 for k in range(10)], dtype=np.int32)
        code, F, st = pgb.pgb_solve_poses([ca, cb], pose_ctx, 0, Rs, ts, pgb.PGB_FP64, 1e-9, 2000, 100)
        assert code == 0
        for k, bodies in ((0, _pair(seed=5, nu=5, nq=20)), (1, _pair(seed=9, nu=7, nq=35))):
            c1 = gpu_context(bodies, lanes=1, **TC)
            refs.append(c1)
            sel = np.nonzero(pose_ctx == k)[0]
            code1, F1, st1 = pgb.pgb_solve_batch(c1, 0, Rs[sel], ts[sel], pgb.PGB_FP64, 1e-9, 2000, 100)
            assert code1 == 0
            np.testing.assert_allclose(F[sel], F1, rtol=1e-9, atol=1e-12)
            assert np.abs(np.array([st[i]["iterations"] for i in sel]) -
                          np.array([s["iterations"] for s in st1])).max() <= 1
        # the molecules differ, so do their energies at one pose
        assert abs(F[0, 1] - F[1, 1]) > 1e-3 * abs(F[0, 1])
    finally:
        for c in [ca, cb] + refs:
            pgb.pgb_destroy(c)


def test_pose_batch_argument_checks():
    c = gpu_context(_pair(), batch=2, **TC)
    try:
        Rs, ts = _poses(3, 2)
        bad = Rs.copy()
        bad[1] = 2 * bad[1]
        with pytest.raises(pgb.PgbError):
            pgb.pgb_solve_batch(c, 0, bad, ts, pgb.PGB_FP64, 1e-8, 100, 50)
        with pytest.raises(pgb.PgbError):
            pgb.pgb_solve_poses([c], np.array([0, 1], dtype=np.int32), 0, Rs, ts, pgb.PGB_FP64, 1e-8, 100, 50)
        with pytest.raises(pgb.PgbError):
            pgb.pgb_solve_poses([c], np.array([0, 0], dtype=np.int32), 5, Rs, ts, pgb.PGB_FP64, 1e-8, 100, 50)
        # 33 poses of 2 bodies exceed the 64 bodies a union holds
        c2 = gpu_context(_pair(), batch=33, **TC)
        try:
            R3, t3 = _poses(4, 33)
            with pytest.raises(pgb.PgbError):
                pgb.pgb_solve_batch(c2, 0, R3, t3, pgb.PGB_FP64, 1e-8, 100, 50)
        finally:
            pgb.pgb_destroy(c2)
    finally:
        pgb.pgb_destroy(c)


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("precond", [0, 1])
def test_replayed_lockstep_iterations_match_host_loop(mode, precond):
    """The lockstep iterations replayed from a graph (graphs = 2: a device
    while loop, per-problem convergence and the body mask of the products on
    the device) reproduce the host-driven loop (graphs = 1) bit for bit, with
    the same iteration counts, through restarts (restart 8) and problems that
    finish at different iterations; the host makes far fewer launch calls."""
    m, tol, _ = MODES[mode]
    Rs, ts = _poses(47, 5)
    ch = gpu_context(_pair(), batch=5, graphs=1, precond=precond, **TC)
    cg = gpu_context(_pair(), batch=5, graphs=2, precond=precond, **TC)
    try:
        pgb.pgb_timing(ch, True, read=False)
        pgb.pgb_timing(cg, True, read=False)
        codeh, Fh, sth = pgb.pgb_solve_batch(ch, 0, Rs, ts, m, tol, 2000, 8)
        codeg, Fg, stg = pgb.pgb_solve_batch(cg, 0, Rs, ts, m, tol, 2000, 8)
        th = pgb.pgb_timing(ch, False, read=True)
        tg = pgb.pgb_timing(cg, False, read=True)
        assert codeh == 0 and codeg == 0
        assert np.array_equal(Fg, Fh)
        assert [s["iterations"] for s in stg] == [s["iterations"] for s in sth]
        assert [s["rel_residual"] for s in stg] == [s["rel_residual"] for s in sth]
        assert tg["host_launches"] < 0.5 * th["host_launches"]
    finally:
        pgb.pgb_destroy(ch)
        pgb.pgb_destroy(cg)


@pytest.mark.parametrize("mode", ["fp32", "refine"])
def test_replayed_iterations_molecules_of_two_sizes(mode):
    """Chunks of two molecules of different sizes (their problems finish at
    different iterations, so the device body mask drops finished ones from
    the products mid-cycle): graphs = 2 equals the host loop bit for bit."""
    m, tol, _ = MODES[mode]
    Rs, ts = _poses(53, 6)
    pose_ctx = np.array([0, 1, 0, 1, 0, 1])
    out = {}
    for gr in (1, 2):
        ctxs = [gpu_context(_pair(nu=5), batch=3, graphs=gr, **TC), gpu_context(_pair(seed=9, nu=7), graphs=gr, **TC)]
        try:
            out[gr] = pgb.pgb_solve_poses(ctxs, pose_ctx, 0, Rs, ts, m, tol, 2000, 100)
        finally:
            for c in ctxs:
                pgb.pgb_destroy(c)
    (c1, F1, s1), (c2, F2, s2) = out[1], out[2]
    assert c1 == 0 and c2 == 0
    assert np.array_equal(F2, F1)
    assert [s["iterations"] for s in s2] == [s["iterations"] for s in s1]

"""Pose batches (pgb_solve_batch, pgb_solve_poses with pgb_params.batch > 1)
against the CPU oracle: every pose's four energies (Eq. 11-16) must match
those of that pose's dense FP64 solve (Section 3.2 GMRES replaced by LU),
across chunks of 3 poses with a padded last chunk and molecules of two mesh
sizes, at theta = 0 (the direct sum, so the only difference is the solve)."""
import numpy as np
import pytest

import synth
from oracle.energy import energies
from problems import gpu_context, oracle_system, star_molecule

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_1506_03745_gb300 as pgb  # noqa: E402

KEYS = ("coulomb", "solvation", "surface", "total")
# FP64 GMRES to 1e-10: energies within 1e-8 of the LU solution; FP32 inner
# iterations with the FP64-class residual to 1e-9: within 1e-6
MODES = {"fp64": (pgb.PGB_FP64, 1e-10, 1e-8), "refine": (pgb.PGB_FP32_REFINE, 1e-9, 1e-6)}


def _surface():
    v, f = synth.icosphere(2, 5.0)
    return dict(kind="sigma", verts=v, tris=f, eps_in=1.0, qxyz=np.zeros((0, 3)), q=np.zeros(0), bc=-0.05,
                R=np.eye(3), t=np.array([15.0, 0.0, 0.0]))


def _pair(nu):
    return [star_molecule(seed=5, nu=nu, nq=20, r0=6.0)[0], _surface()]


def _poses(seed, B):
    Rs = synth.random_rotations(seed, B)
    ts = np.stack([np.array([0.3 * k, -0.2 * k, 0.1 * (k % 3)]) for k in range(B)])
    return Rs, ts


_oracle_cache = {}


def _oracle_energies(nu, R, t):
    key = (nu, tuple(np.round(R, 12).ravel()), tuple(t))
    if key not in _oracle_cache:
        bodies = _pair(nu)
        bodies[0]["R"], bodies[0]["t"] = R, t
        so = oracle_system(bodies, theta=0.0)
        _oracle_cache[key] = energies(so, so.solve())
    return _oracle_cache[key]


def _check(F, want, rel):
    for k, name in enumerate(KEYS):
        assert F[k] == pytest.approx(want[name], rel=rel, abs=1e-10 * abs(want["total"])), name


@pytest.mark.parametrize("mode", sorted(MODES))
def test_solve_batch_matches_oracle_per_pose(mode):
    m, tol, rel = MODES[mode]
    Rs, ts = _poses(51, 4)                      # chunks of 3: [0 1 2] [3 + 2 padding poses]
    ctx = gpu_context(_pair(5), batch=3, theta=0.0)
    try:
        code, F, st = pgb.pgb_solve_batch(ctx, 0, Rs, ts, m, tol, 3000, 100)
        assert code == 0 and len(st) == 4
        for b in range(4):
            assert st[b]["rel_residual"] <= tol
            _check(F[b], _oracle_energies(5, Rs[b], ts[b]), rel)
        assert np.ptp(F[:, 1]) > 1e-6 * abs(F[0, 1])   # the poses differ
    finally:
        pgb.pgb_destroy(ctx)


@pytest.mark.parametrize("mode", sorted(MODES))
def test_solve_poses_two_molecule_sizes_match_oracle(mode):
    m, tol, rel = MODES[mode]
    Rs, ts = _poses(52, 5)
    nus = (4, 5)                                 # 320 and 500 panels
    pose_ctx = np.array([0, 1, 0, 1, 0])         # chunks of 3: [0 1 0] [1 0 + padding]
    ctxs = [gpu_context(_pair(nus[0]), batch=3, theta=0.0), gpu_context(_pair(nus[1]), theta=0.0)]
    try:
        code, F, st = pgb.pgb_solve_poses(ctxs, pose_ctx, 0, Rs, ts, m, tol, 3000, 100)
        assert code == 0 and len(st) == 5
        for b in range(5):
            assert st[b]["rel_residual"] <= tol
            _check(F[b], _oracle_energies(nus[pose_ctx[b]], Rs[b], ts[b]), rel)
    finally:
        for c in ctxs:
            pgb.pgb_destroy(c)

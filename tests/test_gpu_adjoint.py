"""Adjoint path on the GPU (pgb_matvec_transpose, pgb_grad) against the
dense oracle, the dot-product identity and finite differences."""
import numpy as np
import pytest

import synth
from oracle.gradient import gradients
from problems import gpu_context, oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_1506_03745_gb300 as pgb  # noqa: E402


def _bodies(kind="sigma", nu=4, level=2, t=(10.5, 0.4, -0.3)):
    v, f = synth.star_surface(4, nu, 3.5)
    rng = np.random.default_rng(2)
    mol = dict(kind="dielectric", verts=v, tris=f, eps_in=4.0, qxyz=rng.uniform(-1.0, 1.0, size=(6, 3)),
               q=rng.uniform(-1, 1, 6), bc=0.0)
    v2, f2 = synth.icosphere(level, 3.0)
    srf = dict(kind=kind, verts=v2, tris=f2, eps_in=1.0, qxyz=np.zeros((0, 3)), q=np.zeros(0),
               bc=-0.05 if kind == "sigma" else 0.05, R=np.eye(3), t=np.asarray(t, dtype=float))
    return [mol, srf]


def _tmv(ctx, lam, prec):
    lt = torch.tensor(lam, device="cuda")
    yt = torch.empty_like(lt)
    pgb.pgb_matvec_transpose(ctx, lt, yt, prec)
    torch.cuda.synchronize()
    return yt.cpu().numpy()


@pytest.mark.parametrize("kind", ["sigma", "phi"])
def test_transposed_product_matches_dense_transpose(kind):
    bodies = _bodies(kind)
    so = oracle_system(bodies, theta=0.0)
    ctx = gpu_context(bodies, theta=0.0, leaf_size=16)
    try:
        A, _ = so.assemble()
        lam = np.random.default_rng(5).normal(size=so.n)
        ref = A.T @ lam
        scale = np.abs(ref).max()
        assert np.abs(_tmv(ctx, lam, pgb.PGB_FP64) - ref).max() / scale < 1e-11
        assert np.abs(_tmv(ctx, lam, pgb.PGB_FP32) - ref).max() / scale < 5e-6
    finally:
        pgb.pgb_destroy(ctx)


def test_transposed_treecode_accuracy():
    bodies = _bodies("sigma", nu=6, level=3)
    so = oracle_system(bodies, theta=0.0)
    ctx = gpu_context(bodies, theta=0.5, P=6, leaf_size=16)
    try:
        A, _ = so.assemble()
        lam = np.random.default_rng(6).normal(size=so.n)
        ref = A.T @ lam
        for prec in (pgb.PGB_FP64, pgb.PGB_FP32):
            err = np.abs(_tmv(ctx, lam, prec) - ref).max() / np.abs(ref).max()
            assert err < 2e-3
        stats = pgb.pgb_tree_stats(ctx)
        assert stats["n_far"] > 0
    finally:
        pgb.pgb_destroy(ctx)


def test_dot_product_identity_direct_sum():
    bodies = _bodies("phi")
    ctx = gpu_context(bodies, theta=0.0)
    try:
        n = pgb.pgb_num_unknowns(ctx)
        rng = np.random.default_rng(7)
        x, lam = rng.normal(size=n), rng.normal(size=n)
        xt = torch.tensor(x, device="cuda")
        yt = torch.empty_like(xt)
        pgb.pgb_matvec(ctx, xt, yt, pgb.PGB_FP64)
        ax = yt.cpu().numpy()
        atl = _tmv(ctx, lam, pgb.PGB_FP64)
        assert lam @ ax == pytest.approx(atl @ x, rel=1e-12)
    finally:
        pgb.pgb_destroy(ctx)


@pytest.mark.parametrize("kind,theta,P", [("phi", 0.5, 6), ("sigma", 0.6, 3), ("sigma", 0.4, 8)])
def test_transpose_is_exact_for_the_treecode(kind, theta, P):
    """The transposed treecode is the exact transpose of the forward treecode
    product (same near/far split, expansion and corrections):
    <A x, lam> = <x, A^T lam> to rounding for any theta and P."""
    bodies = _bodies(kind, nu=6, level=3)
    ctx = gpu_context(bodies, theta=theta, P=P, leaf_size=8)
    try:
        assert pgb.pgb_tree_stats(ctx)["n_far"] > 0
        n = pgb.pgb_num_unknowns(ctx)
        rng = np.random.default_rng(8)
        x, lam = rng.normal(size=n), rng.normal(size=n)
        xt = torch.tensor(x, device="cuda")
        yt = torch.empty_like(xt)
        pgb.pgb_matvec(ctx, xt, yt, pgb.PGB_FP64)
        lhs = lam @ yt.cpu().numpy()
        rhs = _tmv(ctx, lam, pgb.PGB_FP64) @ x
        assert rhs == pytest.approx(lhs, rel=1e-11)
        x32 = torch.tensor(x, dtype=torch.float32, device="cuda")
        y32 = torch.empty_like(x32)
        pgb.pgb_matvec(ctx, x32, y32, pgb.PGB_FP32)
        assert _tmv(ctx, lam, pgb.PGB_FP32) @ x == pytest.approx(lam @ y32.double().cpu().numpy(), rel=1e-5)
    finally:
        pgb.pgb_destroy(ctx)


def _solve(ctx, tol=1e-11):
    n = pgb.pgb_num_unknowns(ctx)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    code, _ = pgb.pgb_solve(ctx, pgb.PGB_FP64, tol, 3000, 100, x)
    assert code == 0
    return x


@pytest.mark.parametrize("kind", ["sigma", "phi"])
def test_gradients_match_dense_adjoint(kind):
    bodies = _bodies(kind)
    so = oracle_system(bodies, theta=0.0)
    ref = gradients(so)
    ctx = gpu_context(bodies, theta=0.0)
    try:
        x = _solve(ctx)
        code, dq, dbc, dt, st = pgb.pgb_grad(ctx, x, 6, 2, pgb.PGB_FP64, 1e-11, 2000, 100)
        assert code == 0
        np.testing.assert_allclose(dq, ref["dq"][0], rtol=1e-8, atol=1e-10)
        assert dbc[1] == pytest.approx(ref["dbc"][1], rel=1e-8)
        np.testing.assert_allclose(dt, np.array(ref["dt"]), rtol=1e-5, atol=1e-8)
        # Euler's identity of the quadratic form and translation invariance
        e = pgb.pgb_energy(ctx, x)
        bc = bodies[1]["bc"]
        assert bodies[0]["q"] @ dq + bc * dbc[1] == pytest.approx(2 * e["total"], rel=1e-8)
        np.testing.assert_allclose(dt[0], -dt[1], rtol=1e-6, atol=1e-10)
    finally:
        pgb.pgb_destroy(ctx)


def _fd_translation(ctx, bodies, h, frozen):
    """Central differences of the total energy in the surface's translation;
    frozen: the interaction lists of the base pose are kept (reading G20)."""
    t0 = np.asarray(bodies[1]["t"])
    fd = np.zeros(3)
    for ax in range(3):
        f = []
        for sgn in (1, -1):
            tt = t0.copy()
            tt[ax] += sgn * h
            pgb.pgb_set_pose(ctx, 1, np.eye(3), tt)
            if frozen:
                pgb.pgb_tree_refresh(ctx)
            else:
                pgb.pgb_tree_build(ctx)
            f.append(pgb.pgb_energy(ctx, _solve(ctx))["total"])
        fd[ax] = (f[0] - f[1]) / (2 * h)
    pgb.pgb_set_pose(ctx, 1, np.eye(3), t0)
    return fd


@pytest.mark.parametrize("theta,P", [(0.0, 6), (0.5, 8)])
def test_translation_gradient_matches_finite_differences(theta, P):
    """dF/dt of the adjoint (FP64) against central differences with h = 1e-3 A,
    within 1e-4 of the gradient's norm: the direct sum, and the treecode with
    the lists of the base pose held for the displaced solves."""
    bodies = _bodies("sigma", nu=6, level=3)
    ctx = gpu_context(bodies, theta=theta, P=P, leaf_size=16)
    try:
        if theta > 0:
            assert pgb.pgb_tree_stats(ctx)["n_far"] > 0
        x = _solve(ctx)
        code, dq, dbc, dt, st = pgb.pgb_grad(ctx, x, 6, 2, pgb.PGB_FP64, 1e-11, 2000, 100)
        assert code == 0
        fd = _fd_translation(ctx, bodies, 1e-3, frozen=theta > 0)
        assert np.abs(dt[1] - fd).max() <= 1e-4 * np.linalg.norm(fd)
        # the refreshed tree at the base pose gives the base solution back
        pgb.pgb_tree_refresh(ctx)
        assert pgb.pgb_energy(ctx, _solve(ctx))["total"] == pytest.approx(pgb.pgb_energy(ctx, x)["total"], rel=1e-10)
    finally:
        pgb.pgb_destroy(ctx)


def test_translation_gradient_fp32_adjoint():
    """The FP32 adjoint of the FP32 + refinement solve, the same differences
    (treecode, lists held) within 1e-4 of the gradient's norm."""
    bodies = _bodies("sigma", nu=6, level=3)
    ctx = gpu_context(bodies, theta=0.5, P=8, leaf_size=16)
    try:
        n = pgb.pgb_num_unknowns(ctx)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        code, _ = pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, 1e-9, 3000, 100, x)
        assert code == 0
        code, dq, dbc, dt, st = pgb.pgb_grad(ctx, x, 6, 2, pgb.PGB_FP32, 1e-6, 2000, 100)
        assert code == 0
        fd = _fd_translation(ctx, bodies, 1e-3, frozen=True)
        assert np.abs(dt[1] - fd).max() <= 1e-4 * np.linalg.norm(fd)
    finally:
        pgb.pgb_destroy(ctx)


def test_refresh_needs_a_built_tree():
    bodies = _bodies("sigma")
    ctx = gpu_context(bodies, theta=0.5, build=False)
    try:
        with pytest.raises(pgb.PgbError) as ei:
            pgb.pgb_tree_refresh(ctx)
        assert ei.value.code == pgb.PGB_ESTATE
    finally:
        pgb.pgb_destroy(ctx)

"""Block-diagonal (self-term) right preconditioner of GMRES: the solution is
the dense oracle's LU solution, the residual test is unchanged, and it takes
no more iterations than the plain solver; the adjoint solve with the
transposed preconditioner gives the same gradients."""
import numpy as np
import pytest

from oracle.energy import energies
from problems import gpu_context, oracle_system, spheres, star_molecule

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1506_03745_gb300 as pgb  # noqa: E402


def _solve(ctx, mode, tol):
    n = pgb.pgb_num_unknowns(ctx)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    code, st = pgb.pgb_solve(ctx, mode, tol, 2000, 100, x)
    torch.cuda.synchronize()
    return code, st, x


@pytest.mark.parametrize("kind", ["sigma", "phi"])
@pytest.mark.parametrize("mode", ["fp64", "refine"])
def test_preconditioned_solve_matches_dense_oracle(kind, mode):
    bodies = spheres(kind=kind, level_mol=2, level_srf=2)
    so = oracle_system(bodies, theta=0.0)
    xo = so.solve()
    eo = energies(so, xo)
    m = pgb.PGB_FP64 if mode == "fp64" else pgb.PGB_FP32_REFINE
    tol = 1e-11 if mode == "fp64" else 1e-8
    plain = gpu_context(bodies, theta=0.0)
    ctx = gpu_context(bodies, theta=0.0, precond=1)
    try:
        code, st, x = _solve(ctx, m, tol)
        assert code == 0 and st["rel_residual"] <= tol
        xn = x.cpu().numpy()
        assert np.abs(xn - xo).max() / np.abs(xo).max() < (1e-9 if mode == "fp64" else 1e-6)
        e = pgb.pgb_energy(ctx, x)
        for k in ("solvation", "surface", "total"):
            assert e[k] == pytest.approx(eo[k], rel=1e-7 if mode == "fp64" else 1e-6)
        code0, st0, _ = _solve(plain, m, tol)
        assert code0 == 0
        assert st["iterations"] <= st0["iterations"]
    finally:
        pgb.pgb_destroy(ctx)
        pgb.pgb_destroy(plain)


def test_preconditioner_cuts_iterations_on_the_star_molecule():
    bodies = star_molecule(nu=8)
    plain = gpu_context(bodies)
    ctx = gpu_context(bodies, precond=1)
    try:
        c0, s0, x0 = _solve(plain, pgb.PGB_FP64, 1e-8)
        c1, s1, x1 = _solve(ctx, pgb.PGB_FP64, 1e-8)
        assert c0 == 0 and c1 == 0
        assert s1["iterations"] < 0.8 * s0["iterations"]
        e0, e1 = pgb.pgb_energy(plain, x0), pgb.pgb_energy(ctx, x1)
        assert e1["solvation"] == pytest.approx(e0["solvation"], rel=1e-6)
    finally:
        pgb.pgb_destroy(ctx)
        pgb.pgb_destroy(plain)


@pytest.mark.parametrize("kind", ["sigma", "phi"])
def test_preconditioned_adjoint_gives_the_same_gradients(kind):
    bodies = spheres(kind=kind, level_mol=2, level_srf=2)
    out = []
    for pc in (0, 1):
        ctx = gpu_context(bodies, theta=0.0, precond=pc)
        try:
            code, st, x = _solve(ctx, pgb.PGB_FP64, 1e-11)
            assert code == 0
            code, dq, dbc, dt, gst = pgb.pgb_grad(ctx, x, 1, 2, pgb.PGB_FP64, 1e-11, 2000, 100)
            assert code == 0
            out.append((dq, dbc, dt, gst["iterations"]))
        finally:
            pgb.pgb_destroy(ctx)
    (dq0, dbc0, dt0, it0), (dq1, dbc1, dt1, it1) = out
    np.testing.assert_allclose(dq1, dq0, rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(dbc1, dbc0, rtol=1e-8, atol=1e-12)
    np.testing.assert_allclose(dt1, dt0, rtol=1e-6, atol=1e-10)
    assert it1 <= it0


@pytest.mark.parametrize("precond", [0, 1])
def test_overlapped_fp64_residual(precond):
    """FP32 + refinement with the FP64 product of the outer residual started
    early on a side stream (overlap = 1) against the same solve with the FP64
    product of the final iterate (overlap = 0): both meet the tolerance in the
    true FP64 residual, report it, and give the same energies."""
    bodies = spheres(kind="sigma", level_mol=4, level_srf=4)
    out = []
    for ov in (0, 1):
        ctx = gpu_context(bodies, precond=precond, overlap=ov)
        try:
            code, st, x = _solve(ctx, pgb.PGB_FP32_REFINE, 1e-6)
            assert code == 0
            n = pgb.pgb_num_unknowns(ctx)
            b = torch.empty(n, dtype=torch.float64, device="cuda")
            ax = torch.empty_like(b)
            pgb.pgb_rhs(ctx, b)
            pgb.pgb_matvec(ctx, x, ax, pgb.PGB_FP64)
            true_rel = float(torch.linalg.norm(b - ax) / torch.linalg.norm(b))
            assert true_rel <= 1.05e-6
            assert st["rel_residual"] == pytest.approx(true_rel, rel=0.1, abs=3e-8)
            out.append(pgb.pgb_energy(ctx, x))
        finally:
            pgb.pgb_destroy(ctx)
    for k in ("solvation", "surface", "total"):
        assert out[1][k] == pytest.approx(out[0][k], rel=2e-7)

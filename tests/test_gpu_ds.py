"""The double-single FP64-class product (PGB_FP64_DS: P2P and M2P in pairs of
FP32 on the FP32 pipe) against the native FP64 product and the oracle, and
the refinement whose outer residual uses it."""
import numpy as np
import pytest

from oracle.treecode import TreecodeOperator
from problems import gpu_context, oracle_system, spheres, star_molecule

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_1506_03745_gb300 as pgb  # noqa: E402


def _products(ctx, x):
    xt = torch.tensor(x, device="cuda")
    y64 = torch.empty_like(xt)
    yds = torch.empty_like(xt)
    pgb.pgb_matvec(ctx, xt, y64, pgb.PGB_FP64)
    pgb.pgb_matvec(ctx, xt, yds, pgb.PGB_FP64_DS)
    return y64.cpu().numpy(), yds.cpu().numpy()


@pytest.mark.parametrize("case", ["spheres_sigma", "spheres_phi", "star", "kappa0"])
def test_ds_product_matches_fp64(case):
    kappa = 0.0 if case == "kappa0" else 0.125
    if case.startswith("spheres"):
        bodies = spheres(kind="phi" if case == "spheres_phi" else "sigma", level_mol=3, level_srf=3)
    elif case == "star":
        bodies = star_molecule(seed=4, nu=12, nq=40)
    else:
        bodies = spheres(kind="sigma", level_mol=3, level_srf=3)
    ctx = gpu_context(bodies, kappa=kappa, theta=0.5, P=6)
    try:
        n = pgb.pgb_num_unknowns(ctx)
        x = np.random.default_rng(5).normal(size=n)
        y64, yds = _products(ctx, x)
        err = np.abs(yds - y64).max() / np.abs(y64).max()
        assert err < 1e-12, err
    finally:
        pgb.pgb_destroy(ctx)


@pytest.mark.parametrize("P", [0, 3, 8])
def test_ds_product_against_oracle_treecode(P):
    """Every Taylor order (the kernels are instantiated per P) against the
    oracle's treecode, at its FP64 agreement level."""
    bodies = spheres(kind="sigma", level_mol=2, level_srf=2)
    so = oracle_system(bodies, theta=0.5, P=P, leaf_size=8)
    ctx = gpu_context(bodies, theta=0.5, P=P, leaf_size=8)
    try:
        x = np.random.default_rng(6).normal(size=so.n)
        ref = TreecodeOperator(so).apply(x)
        y64, yds = _products(ctx, x)
        assert np.abs(yds - ref).max() / np.abs(ref).max() < 1e-10
        assert np.abs(yds - y64).max() / np.abs(y64).max() < 1e-12
    finally:
        pgb.pgb_destroy(ctx)


@pytest.mark.parametrize("overlap", [0, 1])
def test_refinement_with_ds_residual(overlap):
    """FP32 inner solves with the double-single outer residual reach the
    same energies as with the native FP64 residual, and the reported
    residual is the FP64 residual of the returned x."""
    bodies = spheres(kind="sigma", level_mol=4, level_srf=4)
    out = {}
    for res in (0, 1):
        ctx = gpu_context(bodies, theta=0.5, P=6, residual=res, overlap=overlap)
        try:
            n = pgb.pgb_num_unknowns(ctx)
            x = torch.empty(n, dtype=torch.float64, device="cuda")
            code, st = pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, 1e-8, 2000, 100, x)
            assert code == 0 and st["rel_residual"] <= 1e-8
            b = torch.empty_like(x)
            pgb.pgb_rhs(ctx, b)
            y = torch.empty_like(x)
            pgb.pgb_matvec(ctx, x, y, pgb.PGB_FP64)
            true_rel = float(torch.linalg.norm(b - y) / torch.linalg.norm(b))
            assert true_rel <= 2e-8
            out[res] = pgb.pgb_energy(ctx, x)
        finally:
            pgb.pgb_destroy(ctx)
    for k in ("solvation", "surface", "total"):
        assert out[1][k] == pytest.approx(out[0][k], rel=1e-8)

"""The bounded grid barrier of the fused Arnoldi kernel: a barrier that
nothing completes gives up after its time limit and reports it, and the
context stays usable (a solve afterwards matches the dense oracle)."""
import time

import numpy as np
import pytest

from problems import gpu_context, oracle_system, spheres

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1506_03745_gb300 as pgb  # noqa: E402


def test_barrier_completes_and_times_out():
    assert pgb.pgb_barrier_check(1) == (pgb.PGB_OK, 0)
    t0 = time.perf_counter()
    assert pgb.pgb_barrier_check(2) == (pgb.PGB_OK, 1)
    assert time.perf_counter() - t0 > 0.9
    bodies = spheres(kind="sigma", level_mol=2, level_srf=2)
    so = oracle_system(bodies, theta=0.0)
    ctx = gpu_context(bodies, theta=0.0)
    try:
        n = pgb.pgb_num_unknowns(ctx)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        code, st = pgb.pgb_solve(ctx, pgb.PGB_FP64, 1e-10, 2000, 100, x)
        assert code == 0
        xo = so.solve()
        assert np.abs(x.cpu().numpy() - xo).max() / np.abs(xo).max() < 1e-8
    finally:
        pgb.pgb_destroy(ctx)

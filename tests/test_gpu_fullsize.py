"""The benchmark workload at full size (two spheres, 2 x 20480 panels,
theta 0.5, P 6, leaf 32, K 7) in the launch configuration bench.py times:
sampled rows against the oracle's direct sum, eight sampled target groups
against the oracle's treecode row by row (FP32 and FP64), FP32 against FP64,
and the solve's energies against the dense/analytical expectations."""
import os

import numpy as np
import pytest

from oracle.analytical import interaction
from oracle import units
from problems import fullsize_vectors, gpu_context, oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import bench  # noqa: E402
import paper_1506_03745_gb300 as pgb  # noqa: E402


@pytest.fixture(scope="module")
def full():
    bodies = bench.workload_bodies()
    ctx = gpu_context(bodies, **bench.PARAMS)
    yield bodies, ctx
    pgb.pgb_destroy(ctx)


def test_sampled_rows_match_direct_sum(full):
    bodies, ctx = full
    so = oracle_system(bodies, theta=0.0)
    n = pgb.pgb_num_unknowns(ctx)
    x = np.random.default_rng(11).normal(size=n)
    y = {}
    for prec, dt in ((pgb.PGB_FP32, torch.float32), (pgb.PGB_FP64, torch.float64)):
        xt = torch.tensor(x, dtype=dt, device="cuda")
        yt = torch.empty_like(xt)
        pgb.pgb_matvec(ctx, xt, yt, prec)
        torch.cuda.synchronize()
        y[prec] = yt.double().cpu().numpy()
    # FP32 vs FP64 on the same lists: the precision of the FP32 kernels
    assert np.abs(y[pgb.PGB_FP32] - y[pgb.PGB_FP64]).max() / np.abs(y[pgb.PGB_FP64]).max() < 2e-6
    # sampled rows of both bodies against the exact direct sum (treecode error only)
    N = 20480
    rows = np.r_[np.arange(0, N, 1601), N - 1]
    for a, off in ((0, 0), (1, 2 * N)):
        ref = so.apply_rows(x, a, rows)
        blocks = [y[pgb.PGB_FP64][off + k * N + rows] for k in range(len(ref))]
        for got, want in zip(blocks, ref):
            assert np.abs(got - want).max() / np.abs(want).max() < 5e-4


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize_rows.txt")


def _golden_rows():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#"):
            continue
        name, i, v = line.split()
        out.setdefault(name, ([], []))
        out[name][0].append(int(i))
        out[name][1].append(float(v))
    return {k: (np.array(a), np.array(b)) for k, (a, b) in out.items()}


# bounds on |GPU - oracle treecode| per sampled row: the FP64 product carries
# only rounding (1e-11); the FP32 one the FP32 kernels' rounding (SFU
# rsqrt/ex2 to about 2^-22, FP32 moments and recurrences) on every term
ROW_TOL = {"fp64": 1e-11, "fp32": 2e-6}


def test_sampled_groups_match_oracle_treecode_row_by_row(full):
    """Eight target groups (256 targets; tests/golden/fullsize_rows.txt from
    make_fullsize_rows.py, oracle/ only).  Positive densities: every row is a
    sum of terms of one sign (up to the near-field corrections), so each row
    is held to a relative bound of its own.  Normal densities: rows with
    cancellation, held relative to the largest sampled row of their block."""
    bodies, ctx = full
    n = pgb.pgb_num_unknowns(ctx)
    N = 20480
    ref = _golden_rows()
    vecs = fullsize_vectors(n)
    for name, (idx, want) in ref.items():
        assert len(idx) == 8 * 32 * 3 // 2          # 4 molecule groups x 2 rows + 4 surface groups
        for prec, dt, key in ((pgb.PGB_FP32, torch.float32, "fp32"), (pgb.PGB_FP64, torch.float64, "fp64")):
            xt = torch.tensor(vecs[name], dtype=dt, device="cuda")
            yt = torch.empty_like(xt)
            pgb.pgb_matvec(ctx, xt, yt, prec)
            torch.cuda.synchronize()
            got = yt.double().cpu().numpy()[idx]
            err = np.abs(got - want)
            if name == "positive":
                assert np.all(err <= ROW_TOL[key] * np.abs(want)), (key, (err / np.abs(want)).max())
            else:
                for lo, hi in ((0, N), (N, 2 * N), (2 * N, 3 * N)):
                    blk = (idx >= lo) & (idx < hi)
                    assert np.all(err[blk] <= ROW_TOL[key] * np.abs(want[blk]).max()), (key, lo)


def test_full_size_solve_energy_is_close_to_analytical(full):
    bodies, ctx = full
    n = pgb.pgb_num_unknowns(ctx)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    code, st = pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, 1e-6, 2000, 100, x)
    assert code == 0 and st["rel_residual"] <= 1e-6
    e = pgb.pgb_energy(ctx, x, 2)
    _, parts = interaction(4, 4, 12, 1, 4, 80, 0.125, sigma0=units.sigma_from_c_m2(0.05))
    # level-5 meshes: discretisation error ~ 1/N (level 3 was 0.3 %)
    assert e["solvation"] == pytest.approx(parts["solv"], rel=2e-3)
    assert e["surface"] == pytest.approx(parts["surf"], rel=2e-3)

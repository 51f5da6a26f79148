"""Adjoint gradients of the differentiation workload's coarse version (star
molecule of 2000 panels and 900 charges, 10 A from a 40 A sphere of 3380
panels with sigma0 = -0.05 C/m^2) against the dense FP64 oracle's adjoint
(tests/golden/config4_coarse_gradient.txt, written by
make_config4_coarse_gradient.py from oracle/ alone): the direct sum in FP64,
and the treecode (theta 0.5, P 6) in FP32 + refinement with the FP32 adjoint."""
import os

import numpy as np
import pytest

from problems import config4_coarse, gpu_context

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_1506_03745_gb300 as pgb  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config4_coarse_gradient.txt")


def _golden():
    e, dq, dt, dbc = {}, {}, {}, None
    for line in open(GOLDEN):
        if line.startswith("#"):
            continue
        w = line.split()
        if w[0] == "energy":
            e[w[1]] = float(w[2])
        elif w[0] == "dbc":
            dbc = float(w[2])
        elif w[0] == "dt":
            dt[int(w[1])] = np.array([float(v) for v in w[2:5]])
        elif w[0] == "dq":
            dq[int(w[1])] = float(w[2])
    return e, np.array([dq[k] for k in range(len(dq))]), dbc, np.stack([dt[0], dt[1]])


# (theta, P, solve mode, solve tol, adjoint precision, adjoint tol, bounds on
#  energies, dq, dsigma, dt relative to the oracle's scale)
CASES = {
    "direct_fp64": (0.0, 6, pgb.PGB_FP64, 1e-11, pgb.PGB_FP64, 1e-11, 1e-8, 1e-7, 1e-7, 1e-5),
    "treecode_fp32_refine": (0.5, 6, pgb.PGB_FP32_REFINE, 1e-6, pgb.PGB_FP32, 1e-6, 1e-3, 1e-3, 1e-3, 1e-3),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_config4_coarse_gradients_match_dense_oracle(case):
    theta, P, mode, tol, gprec, gtol, re, rq, rs, rt = CASES[case]
    e_ref, dq_ref, dbc_ref, dt_ref = _golden()
    bodies = config4_coarse()
    assert len(dq_ref) == len(bodies[0]["q"]) == 900
    ctx = gpu_context(bodies, theta=theta, P=P)
    try:
        n = pgb.pgb_num_unknowns(ctx)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        code, st = pgb.pgb_solve(ctx, mode, tol, 3000, 100, x)
        assert code == 0
        e = pgb.pgb_energy(ctx, x)
        for k in ("coulomb", "solvation", "surface", "total"):
            assert e[k] == pytest.approx(e_ref[k], rel=re), k
        code, dq, dbc, dt, ast = pgb.pgb_grad(ctx, x, 900, 2, gprec, gtol, 3000, 100)
        assert code == 0
        assert np.abs(dq - dq_ref).max() <= rq * np.abs(dq_ref).max()
        assert dbc[1] == pytest.approx(dbc_ref, rel=rs)
        assert np.abs(dt - dt_ref).max() <= rt * np.linalg.norm(dt_ref[0])
    finally:
        pgb.pgb_destroy(ctx)

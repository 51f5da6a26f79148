"""pgb_autotune: the chosen parameters come from the candidate set, meet the
accuracy target against the reference candidate and are the fastest such."""
import pytest

from problems import gpu_context, spheres

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_1506_03745_gb300 as pgb  # noqa: E402


def test_autotune_picks_fastest_accurate_candidate():
    ctx = gpu_context(spheres(kind="sigma", level_mol=4, level_srf=4), theta=0.5, P=6)
    try:
        thetas, Ps, leaves = [0.3, 0.5, 0.7], [4, 6], [16, 32]
        chosen, rep = pgb.pgb_autotune(ctx, thetas, Ps, leaves, reps=3, tol=1e-6, target_rel_err=1e-4)
        assert chosen["theta"] in thetas and chosen["P"] in Ps and chosen["leaf_size"] in leaves
        ok = rep[:, 2] <= 1e-4
        assert ok.any()
        k = [(t, p, l) for t in thetas for p in Ps for l in leaves].index(
            (chosen["theta"], chosen["P"], chosen["leaf_size"]))
        assert ok[k] and rep[k, 1] == rep[ok, 1].min()
        assert rep[0, 2] == 0.0 or min(rep[:, 2]) == 0.0   # the reference itself
        # the work-item sizes come from their own candidate set
        assert chosen["p2p_item"] in (16, 32, 64, 128) and chosen["m2p_item"] in (16, 32, 64, 128)
        # the context is usable with the chosen parameters
        n = pgb.pgb_num_unknowns(ctx)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        code, _ = pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, 1e-6, 2000, 100, x)
        assert code == 0
    finally:
        pgb.pgb_destroy(ctx)

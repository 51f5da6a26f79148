"""The paper's grid-convergence case (Section 5.1, Table 1 parameters: far
rule 3 points, close-by rule 37 points, 9 Gauss points per edge in-element,
N_crit 300, P 15, theta 0.5, GMRES tol 1e-9): spheres r = 5 A (eps 4, central
unit charge) and r = 4 A held at phi0 = 1 internal unit, 12 A apart, kappa
0.125, eps 80.  The interaction energy of Eq. 17 approaches the analytical
value of Section 4 (tests/golden/two_sphere_analytical.txt, from the oracle's
series solution) at first order in 1/N, as the paper observes (1.007)."""
import math
import os

import numpy as np
import pytest

import synth
from problems import gpu_context

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_1506_03745_gb300 as pgb  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "two_sphere_analytical.txt")


def _analytical():
    volt, F = None, None
    for line in open(GOLDEN):
        if line.startswith("# one internal potential unit"):
            volt = float(line.split("=")[1].split()[0])
        elif line.split()[:2] == ["paper_5_4_phi1", "60"]:
            F = float(line.split()[2])
    return F, volt


def _f_int(level, volt):
    vm, fm = synth.icosphere(level, 5.0)
    vs, fs = synth.icosphere(level, 4.0)
    mol = dict(kind="dielectric", verts=vm, tris=fm, eps_in=4.0, qxyz=np.zeros((1, 3)), q=np.array([1.0]), bc=0.0)
    srf = dict(kind="phi", verts=vs + np.array([12.0, 0.0, 0.0]), tris=fs, eps_in=1.0, qxyz=np.zeros((0, 3)),
               q=np.zeros(0), bc=volt)
    prm = dict(K=3, K_near=37, n_edge=9, leaf_size=300, P=15, theta=0.5)
    e = {}
    for name, bodies in (("pair", [mol, srf]), ("molecule", [mol]), ("surface", [srf])):
        ctx = gpu_context(bodies, **prm)
        try:
            x = torch.empty(pgb.pgb_num_unknowns(ctx), dtype=torch.float64, device="cuda")
            code, st = pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, 1e-9, 3000, 100, x)
            assert code == 0 and st["rel_residual"] <= 1e-9
            e[name] = pgb.pgb_energy(ctx, x)
        finally:
            pgb.pgb_destroy(ctx)
    return (e["pair"]["solvation"] + e["pair"]["surface"]) - e["molecule"]["solvation"] - e["surface"]["surface"]


def test_paper_two_sphere_case_converges_at_first_order():
    F_an, volt = _analytical()
    errs = [abs(_f_int(level, volt) - F_an) / abs(F_an) for level in (3, 4, 5)]
    orders = [math.log(errs[k] / errs[k + 1]) / math.log(4.0) for k in range(2)]
    assert errs[-1] < 2e-3
    for p in orders:
        assert 0.9 < p < 1.1, orders

"""Nested interfaces on the GPU (pgb_set_region: Stern layers, solvent-filled
cavities) against the oracle's per-region rows (oracle/regions.py)."""
import numpy as np
import pytest

import synth
from oracle import units
from oracle.bem import DIELECTRIC, SET_CHARGE, Body, Params
from oracle.regions import RegionSystem, stern_sphere_solvation
from problems import gpu_context

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_1506_03745_gb300 as pgb  # noqa: E402


def _sphere(level, r, center=(0.0, 0.0, 0.0)):
    v, f = synth.icosphere(level, r)
    return v + np.asarray(center), f


def _mol(level, r, charges, q, eps_in=4.0, center=(0.0, 0.0, 0.0)):
    v, f = _sphere(level, r, center)
    return dict(kind="dielectric", verts=v, tris=f, eps_in=eps_in, qxyz=np.asarray(charges, float),
                q=np.asarray(q, float), bc=0.0)


def _shell(level, r, eps_in, parent=-1, kappa_in=0.0, center=(0.0, 0.0, 0.0)):
    v, f = _sphere(level, r, center)
    return dict(kind="dielectric", verts=v, tris=f, eps_in=eps_in, qxyz=np.zeros((0, 3)), q=np.zeros(0), bc=0.0,
                parent=parent, kappa_in=kappa_in)


def _charged_sphere(level, r, center, sigma):
    v, f = _sphere(level, r, center)
    return dict(kind="sigma", verts=v, tris=f, eps_in=1.0, qxyz=np.zeros((0, 3)), q=np.zeros(0), bc=sigma)


def _oracle(bodies, kappa):
    ob = []
    for b in bodies:
        if b["kind"] == "dielectric":
            ob.append(Body(DIELECTRIC, b["verts"], b["tris"], eps_in=b["eps_in"], charge_xyz=b["qxyz"],
                           charge_q=b["q"]))
        else:
            ob.append(Body(SET_CHARGE, b["verts"], b["tris"], bc_value=units.sigma_from_c_m2(b["bc"])))
    parent = [b.get("parent", -1) for b in bodies]
    kin = [b.get("kappa_in", 0.0) for b in bodies]
    return RegionSystem(ob, 80.0, kappa, parent=parent, kappa_in=kin, params=Params())


def _stern(kappa_in_shell=0.0):
    m = _mol(2, 4.0, [[0.6, -0.3, 0.2], [-0.8, 0.4, 0.0]], [1.0, -0.4])
    m["parent"] = 1
    return [m, _shell(2, 6.0, 80.0, kappa_in=kappa_in_shell)]


def _cavity():
    m = _mol(2, 6.0, [[4.0, 0.0, 0.0], [-3.0, 1.0, 0.5]], [1.0, 0.5])
    return [m, _shell(1, 2.0, 80.0, parent=0)]


def _stern_near_surface():
    bodies = _stern()
    bodies.append(_charged_sphere(2, 4.0, (14.0, 0.0, 0.0), -0.05))
    return bodies


CASES = {"stern": _stern, "cavity": _cavity, "stern_and_surface": _stern_near_surface}


@pytest.mark.parametrize("case", sorted(CASES))
def test_product_and_rhs_match_dense_rows(case):
    """theta = 0: the GPU's region passes are the direct sum, so A x and the
    right-hand side equal the oracle's dense per-region rows."""
    bodies = CASES[case]()
    so = _oracle(bodies, 0.125)
    A, rhs = so.assemble()
    ctx = gpu_context(bodies, theta=0.0)
    try:
        n = pgb.pgb_num_unknowns(ctx)
        assert n == so.n
        x = np.random.default_rng(3).normal(size=n)
        xt = torch.tensor(x, device="cuda")
        y = torch.empty_like(xt)
        pgb.pgb_matvec(ctx, xt, y, pgb.PGB_FP64)
        ref = A @ x
        assert np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-10
        yds = torch.empty_like(xt)
        pgb.pgb_matvec(ctx, xt, yds, pgb.PGB_FP64_DS)
        assert np.abs(yds.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-10
        y32 = torch.empty(n, dtype=torch.float32, device="cuda")
        pgb.pgb_matvec(ctx, xt.float(), y32, pgb.PGB_FP32)
        assert np.abs(y32.double().cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-5
        b = torch.empty_like(xt)
        pgb.pgb_rhs(ctx, b)
        assert np.abs(b.cpu().numpy() - rhs).max() / np.abs(rhs).max() < 1e-10
    finally:
        pgb.pgb_destroy(ctx)


@pytest.mark.parametrize("case", sorted(CASES))
def test_energies_match_dense_solution(case):
    bodies = CASES[case]()
    so = _oracle(bodies, 0.125)
    eo = so.energies(so.solve())
    # a Stern shell has the same permittivity on both sides, so its two rows
    # differ only through the screening: the system is less well conditioned
    # than Eq. 6/7 and the solves stop at tolerances the energies need
    runs = ((0.0, 1e-6, pgb.PGB_FP64, 1e-9, 1), (0.5, 2e-3, pgb.PGB_FP32_REFINE, 1e-6, 1),
            (0.5, 2e-3, pgb.PGB_FP32_REFINE, 1e-6, 0))
    for theta, tol, mode, stol, overlap in runs:  # overlap 1: the FP64 product on a side stream
        ctx = gpu_context(bodies, theta=theta, P=6, overlap=overlap)
        try:
            n = pgb.pgb_num_unknowns(ctx)
            x = torch.empty(n, dtype=torch.float64, device="cuda")
            code, st = pgb.pgb_solve(ctx, mode, stol, 2000, 100, x)
            assert code == 0, st
            e = pgb.pgb_energy(ctx, x)
            for k in ("solvation", "surface", "total"):
                assert e[k] == pytest.approx(eo[k], rel=tol, abs=1e-9)
        finally:
            pgb.pgb_destroy(ctx)


def test_stern_layer_closed_form_on_gpu():
    """Central charge, Stern shell 4 -> 6 A: the GPU treecode solve reaches
    the closed form to the meshes' discretisation error, and the salt term
    E(kappa) - E(0) to 3 %."""
    def solv(kappa):
        m = _mol(3, 4.0, [[0.0, 0.0, 0.0]], [1.0])
        m["parent"] = 1
        ctx = gpu_context([m, _shell(3, 6.0, 80.0)], kappa=kappa, theta=0.5, P=6)
        try:
            x = torch.empty(pgb.pgb_num_unknowns(ctx), dtype=torch.float64, device="cuda")
            code, st = pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, 1e-6, 2000, 100, x)
            assert code == 0, st
            return pgb.pgb_energy(ctx, x)["solvation"]
        finally:
            pgb.pgb_destroy(ctx)
    e5, e0 = solv(0.5), solv(0.0)
    exact = stern_sphere_solvation(1.0, 4.0, 6.0, 4.0, 80.0, 0.5)
    assert e5 == pytest.approx(exact, rel=0.02)
    assert (e5 - e0) == pytest.approx(exact - stern_sphere_solvation(1.0, 4.0, 6.0, 4.0, 80.0, 0.0), rel=0.03)


def test_region_argument_checks():
    bodies = _stern()
    ctx = gpu_context(bodies, theta=0.5)
    try:
        with pytest.raises(pgb.PgbError):
            pgb.pgb_set_region(ctx, 1, 0, 0.0)       # cycle: 0 is inside 1
        with pytest.raises(pgb.PgbError):
            pgb.pgb_set_region(ctx, 0, 0, 0.0)       # its own parent
        with pytest.raises(pgb.PgbError):
            pgb.pgb_set_region(ctx, 0, 1, 0.1)       # screened interior with charges
        with pytest.raises(pgb.PgbError):
            pgb.pgb_set_region(ctx, 1, -1, -1.0)
        n = pgb.pgb_num_unknowns(ctx)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        with pytest.raises(pgb.PgbError):
            pgb.pgb_grad(ctx, x, 2, 2)
        with pytest.raises(pgb.PgbError):
            pgb.pgb_energy_noalloc(ctx, x)
    finally:
        pgb.pgb_destroy(ctx)
    srf = _charged_sphere(1, 3.0, (12.0, 0, 0), 0.05)
    c2 = gpu_context([_mol(1, 4.0, [[0.0, 0, 0]], [1.0]), srf], theta=0.5)
    try:
        with pytest.raises(pgb.PgbError):
            pgb.pgb_set_region(c2, 1, 0, 0.0)        # imposed-value surfaces stay in the solvent
        with pytest.raises(pgb.PgbError):
            pgb.pgb_set_region(c2, 0, 1, 0.0)        # a parent must be dielectric
    finally:
        pgb.pgb_destroy(c2)

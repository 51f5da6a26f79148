"""The energy entry point that allocates no device memory
(pgb_energy_noalloc) against pgb_energy.

Some callers cannot call cudaMalloc: code running under a fixed device-memory
budget or a pool that owns the whole device, and latency-bound loops where an
allocation would synchronise the device.  pgb_energy_noalloc keeps its scratch
in a fixed static device array instead.  This file is collected last so that a
failure here leaves every other test already run."""
import numpy as np
import pytest

from problems import gpu_context, spheres, star_molecule

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_1506_03745_gb300 as pgb  # noqa: E402


def _solved(bodies):
    ctx = gpu_context(bodies, theta=0.5, P=4)
    n = pgb.pgb_num_unknowns(ctx)
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    code, _ = pgb.pgb_solve(ctx, pgb.PGB_FP64, 1e-8, 1000, 100, x)
    assert code == 0
    return ctx, x


@pytest.mark.parametrize("which", ["star_molecule", "molecule_and_surface"])
def test_noalloc_energy_matches_pgb_energy_twice(which):
    bodies = star_molecule(nu=6, nq=40) if which == "star_molecule" else spheres(kind="phi", level_mol=2, level_srf=2)
    ctx, x = _solved(bodies)
    try:
        ref = pgb.pgb_energy(ctx, x)
        for _ in range(2):   # the shared scratch keeps the last call's contents
            got = pgb.pgb_energy_noalloc(ctx, x)
            for k in ("coulomb", "solvation", "surface", "total"):
                assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-14), k
        # a second, different solution through the same scratch
        x2 = 0.5 * x
        ref2 = pgb.pgb_energy(ctx, x2)
        got2 = pgb.pgb_energy_noalloc(ctx, x2)
        for k in ("solvation", "surface", "total"):
            assert got2[k] == pytest.approx(ref2[k], rel=1e-12, abs=1e-14), k
    finally:
        pgb.pgb_destroy(ctx)


def test_noalloc_energy_makes_no_allocation():
    """The library's allocation counter does not move across calls of the
    no-alloc entry point (after its first call on the device, which only looks
    up the static array's address), while a tree rebuild does move it."""
    ctx, x = _solved(spheres(kind="sigma", level_mol=2, level_srf=2))
    try:
        pgb.pgb_energy_noalloc(ctx, x)
        n0 = pgb.pgb_alloc_count()
        for _ in range(3):
            pgb.pgb_energy_noalloc(ctx, x)
        torch.cuda.synchronize()
        assert pgb.pgb_alloc_count() == n0
        pgb.pgb_tree_reset(ctx)
        pgb.pgb_tree_build(ctx)
        assert pgb.pgb_alloc_count() > n0
    finally:
        pgb.pgb_destroy(ctx)


def test_noalloc_rejects_too_many_charges():
    import synth
    v, f = synth.icosphere(1, 20.0)
    nq = pgb.PGB_NOALLOC_MAX_CHARGES + 1
    rng = np.random.default_rng(0)
    xyz = rng.uniform(-5, 5, size=(nq, 3))
    bodies = [dict(kind="dielectric", verts=v, tris=f, eps_in=4.0, qxyz=xyz, q=rng.uniform(-1, 1, nq), bc=0.0)]
    ctx = gpu_context(bodies, theta=0.0)
    try:
        x = torch.zeros(pgb.pgb_num_unknowns(ctx), dtype=torch.float64, device="cuda")
        with pytest.raises(pgb.PgbError) as ei:
            pgb.pgb_energy_noalloc(ctx, x)
        assert ei.value.code == pgb.PGB_EINVAL
        assert "at most" in str(ei.value)
    finally:
        pgb.pgb_destroy(ctx)

"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle."""
import numpy as np
import pytest

import synth

from oracle.energy import energies
from oracle.treecode import TreecodeOperator
from problems import gpu_context, oracle_system, spheres, star_molecule

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import paper_1506_03745_gb300 as pgb  # noqa: E402


def _matvec(ctx, x, prec):
    dt = torch.float32 if prec == pgb.PGB_FP32 else torch.float64
    xt = torch.tensor(x, dtype=dt, device="cuda")
    yt = torch.empty_like(xt)
    pgb.pgb_matvec(ctx, xt, yt, prec)
    torch.cuda.synchronize()
    return yt.double().cpu().numpy()


CASES = {
    "molecule_only": dict(surface=False, level_mol=3),
    "sigma_pair": dict(kind="sigma", level_mol=2, level_srf=2),
    "phi_pair": dict(kind="phi", level_mol=2, level_srf=1, r_srf=3.0, sep=9.0),
    "ragged_geodesic": dict(kind="sigma", mol_nu=5, level_srf=1, sep=10.0),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_direct_sum_matvec_matches_oracle(case):
    bodies = spheres(**CASES[case])
    so = oracle_system(bodies, theta=0.0)
    ctx = gpu_context(bodies, theta=0.0, leaf_size=16)
    try:
        x = np.random.default_rng(1).normal(size=so.n)
        ref = so.apply(x)
        scale = np.abs(ref).max()
        y64 = _matvec(ctx, x, pgb.PGB_FP64)
        assert np.abs(y64 - ref).max() / scale < 1e-11
        y32 = _matvec(ctx, x, pgb.PGB_FP32)
        assert np.abs(y32 - ref).max() / scale < 2e-6
    finally:
        pgb.pgb_destroy(ctx)


@pytest.mark.parametrize("case,theta,P", [("sigma_pair", 0.5, 6), ("phi_pair", 0.6, 3), ("molecule_only", 0.5, 4)])
def test_treecode_matches_oracle_treecode(case, theta, P):
    kw = dict(CASES[case])
    if case == "molecule_only":
        kw["level_mol"] = 2
    bodies = spheres(**kw)
    so = oracle_system(bodies, theta=theta, P=P, leaf_size=8)
    ctx = gpu_context(bodies, theta=theta, P=P, leaf_size=8)
    try:
        tc = TreecodeOperator(so)
        # identical ordering and interaction lists (integer work: bit-exact)
        perm, noff, near, foff, far = pgb.pgb_tree_export(ctx)
        offs = np.cumsum([0] + [p.N for p in so.panels])
        operm = np.concatenate([tr.perm + o for tr, o in zip(tc.trees, offs[:-1])])
        assert np.array_equal(perm, operm)
        node_base = _node_ids(tc)
        assert len(noff) - 1 == len(tc.groups)
        for gi in range(len(tc.groups)):
            on, of = [], []
            for b in range(len(so.bodies)):
                n_, f_ = tc.lists[(gi, b)]
                on += [node_base[b][i] for i in n_]
                of += [node_base[b][i] for i in f_]
            assert sorted(near[noff[gi]:noff[gi + 1]]) == sorted(on)
            assert sorted(far[foff[gi]:foff[gi + 1]]) == sorted(of)
        x = np.random.default_rng(2).normal(size=so.n)
        ref = tc.apply(x)
        scale = np.abs(ref).max()
        y64 = _matvec(ctx, x, pgb.PGB_FP64)
        assert np.abs(y64 - ref).max() / scale < 1e-10
        y32 = _matvec(ctx, x, pgb.PGB_FP32)
        assert np.abs(y32 - ref).max() / scale < 5e-6
    finally:
        pgb.pgb_destroy(ctx)


@pytest.mark.parametrize("items", [(1, 1), (3, 5)])
def test_work_items_split_groups(items):
    """Groups cut into many P2P / M2P work items (down to one tile or one far
    node per block) give the oracle treecode's product."""
    bodies = spheres(**CASES["sigma_pair"])
    so = oracle_system(bodies, theta=0.5, P=6, leaf_size=8)
    ctx = gpu_context(bodies, theta=0.5, P=6, leaf_size=8, p2p_item=items[0], m2p_item=items[1])
    ref_ctx = gpu_context(bodies, theta=0.5, P=6, leaf_size=8)
    try:
        x = np.random.default_rng(5).normal(size=so.n)
        ref = TreecodeOperator(so).apply(x)
        scale = np.abs(ref).max()
        y64 = _matvec(ctx, x, pgb.PGB_FP64)
        assert np.abs(y64 - ref).max() / scale < 1e-10
        assert np.abs(y64 - _matvec(ref_ctx, x, pgb.PGB_FP64)).max() / scale < 1e-13
        y32 = _matvec(ctx, x, pgb.PGB_FP32)
        assert np.abs(y32 - ref).max() / scale < 5e-6
    finally:
        pgb.pgb_destroy(ctx)
        pgb.pgb_destroy(ref_ctx)


def _node_ids(tc):
    """Map oracle per-body DFS node indices to the library's level-order ids
    (roots first, then each level's children in parent order, key order)."""
    levels = []
    for b, tr in enumerate(tc.trees):
        levels.append([(b, 0)])
    ids = [dict() for _ in tc.trees]
    cur = [(b, 0) for b in range(len(tc.trees))]
    nid = 0
    while cur:
        nxt = []
        for b, i in cur:
            ids[b][i] = nid
            nid += 1
        for b, i in cur:
            nxt += [(b, ch) for ch in tc.trees[b].nodes[i]["children"]]
        cur = nxt
    return ids


@pytest.mark.parametrize("kind", ["sigma", "phi"])
@pytest.mark.parametrize("mode", ["fp64", "refine"])
def test_solve_and_energies_match_dense_oracle(kind, mode):
    bodies = spheres(kind=kind, level_mol=2, level_srf=2)
    so = oracle_system(bodies, theta=0.0)
    ctx = gpu_context(bodies, theta=0.0)
    try:
        n = pgb.pgb_num_unknowns(ctx)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        m = pgb.PGB_FP64 if mode == "fp64" else pgb.PGB_FP32_REFINE
        code, st = pgb.pgb_solve(ctx, m, 1e-10, 2000, 100, x)
        assert code == 0 and st["rel_residual"] <= 1e-10
        xo = so.solve()
        assert np.abs(x.cpu().numpy() - xo).max() / np.abs(xo).max() < 1e-8
        e = pgb.pgb_energy(ctx, x, 2)
        eo = energies(so, xo)
        for k in ("coulomb", "solvation", "surface", "total"):
            assert e[k] == pytest.approx(eo[k], rel=1e-8, abs=1e-12)
    finally:
        pgb.pgb_destroy(ctx)


def test_star_molecule_charges_and_rhs():
    bodies = star_molecule(nu=6, nq=40)
    so = oracle_system(bodies, theta=0.0)
    ctx = gpu_context(bodies, theta=0.0)
    try:
        n = pgb.pgb_num_unknowns(ctx)
        b = torch.empty(n, dtype=torch.float64, device="cuda")
        pgb.pgb_rhs(ctx, b)
        _, bo = so.assemble()
        assert np.abs(b.cpu().numpy() - bo).max() / np.abs(bo).max() < 1e-12
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        code, st = pgb.pgb_solve(ctx, pgb.PGB_FP64, 1e-10, 2000, 100, x)
        assert code == 0
        e = pgb.pgb_energy(ctx, x)
        eo = energies(so, so.solve())
        assert e["coulomb"] == pytest.approx(eo["coulomb"], rel=1e-12)
        assert e["solvation"] == pytest.approx(eo["solvation"], rel=1e-8)
    finally:
        pgb.pgb_destroy(ctx)


def test_state_and_argument_errors():
    ctx = pgb.pgb_create(pgb.default_params(), torch.cuda.current_stream())
    try:
        x = torch.zeros(4, dtype=torch.float64, device="cuda")
        assert pgb.lib().pgb_tree_build(ctx) == pgb.PGB_ESTATE
        import synth
        v, f = synth.icosphere(1, 2.0)
        bad = f.copy()
        bad[0, 0] = 10_000
        with pytest.raises(pgb.PgbError) as ei:
            pgb.pgb_mesh_load(ctx, pgb.PGB_DIELECTRIC, v, bad, 4.0)
        assert ei.value.code == pgb.PGB_EINVAL
        vnan = v.copy()
        vnan[3, 1] = np.nan
        with pytest.raises(pgb.PgbError):
            pgb.pgb_mesh_load(ctx, pgb.PGB_DIELECTRIC, vnan, f, 4.0)
        with pytest.raises(pgb.PgbError):
            pgb.pgb_set_solvent(ctx, 80.0, -1.0)
        pgb.pgb_mesh_load(ctx, pgb.PGB_DIELECTRIC, v, f, 4.0)
        st = pgb.lib().pgb_matvec(ctx, x.data_ptr(), x.data_ptr(), pgb.PGB_FP64)
        assert st == pgb.PGB_ESTATE
    finally:
        pgb.pgb_destroy(ctx)


@pytest.mark.parametrize("kind", ["sigma", "phi"])
def test_treecode_energies_within_1e3_of_dense(kind):
    """theta 0.5, P 6 treecode with FP32+refinement against the dense FP64
    oracle: energies within 1e-3 relative."""
    bodies = spheres(kind=kind, level_mol=3, level_srf=3)
    so = oracle_system(bodies, theta=0.0)
    ctx = gpu_context(bodies, theta=0.5, P=6, leaf_size=32)
    try:
        n = pgb.pgb_num_unknowns(ctx)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        code, st = pgb.pgb_solve(ctx, pgb.PGB_FP32_REFINE, 1e-6, 2000, 100, x)
        assert code == 0
        e = pgb.pgb_energy(ctx, x, 2)
        eo = energies(so, so.solve())
        assert e["solvation"] == pytest.approx(eo["solvation"], rel=1e-3)
        assert e["surface"] == pytest.approx(eo["surface"], rel=1e-3)
        assert e["total"] == pytest.approx(eo["total"], rel=1e-3)
    finally:
        pgb.pgb_destroy(ctx)


def test_morton_order_and_lists_at_size():
    """Multi-tile radix sort and warp-parallel traversals: the permutation and
    the interaction-list sizes of the 2 x 20480-panel workload match the oracle."""
    from oracle.treecode import BodyTree, interaction_lists
    import bench
    bodies = bench.workload_bodies()
    so = oracle_system(bodies, theta=0.5, P=6, leaf_size=32)
    ctx = gpu_context(bodies, theta=0.5, P=6, leaf_size=32)
    try:
        perm, noff, near, foff, far = pgb.pgb_tree_export(ctx)
        trees = [BodyTree(b, pn, 7, 32) for b, pn in zip(so.bodies, so.panels)]
        operm = np.concatenate([trees[0].perm, trees[1].perm + so.panels[0].N])
        assert np.array_equal(perm, operm)
        g = 0
        for a, (tr, pn) in enumerate(zip(trees, so.panels)):
            for g0 in range(0, pn.N, 32):
                if g % 97 == 0:   # sampled groups
                    idx = tr.perm[g0:g0 + 32]
                    x = pn.c[idx]
                    nn = sum(len(interaction_lists(tb, x.min(0), x.max(0), 0.5)[0]) for tb in trees)
                    nf = sum(len(interaction_lists(tb, x.min(0), x.max(0), 0.5)[1]) for tb in trees)
                    assert noff[g + 1] - noff[g] == nn and foff[g + 1] - foff[g] == nf
                g += 1
    finally:
        pgb.pgb_destroy(ctx)


def test_upward_graph_replay_matches_plain_launches():
    """The upward pass replayed as a CUDA graph gives bit-identical products
    and right-hand sides to plain launches, across a pose change (graph
    reused: same octree) and a full rebuild (graph recaptured)."""
    bodies = spheres(**CASES["sigma_pair"])
    cg = gpu_context(bodies, theta=0.5, P=5, leaf_size=8, graphs=1)
    cp = gpu_context(bodies, theta=0.5, P=5, leaf_size=8, graphs=0)
    try:
        n = pgb.pgb_num_unknowns(cg)
        x = np.random.default_rng(9).normal(size=n)
        for step in range(3):
            if step == 1:
                R = synth.random_rotations(1, 4)[0]
                t = np.array([12.5, 1.0, -0.5]) - R @ np.array([12.0, 0.0, 0.0])  # keep the centre 12.5 A away
                for c in (cg, cp):
                    pgb.pgb_set_pose(c, 1, R, t)
                    pgb.pgb_tree_build(c)
            if step == 2:
                for c in (cg, cp):
                    pgb.pgb_tree_reset(c)
                    pgb.pgb_tree_build(c)
            for prec in (pgb.PGB_FP32, pgb.PGB_FP64):
                assert np.array_equal(_matvec(cg, x, prec), _matvec(cp, x, prec))
            bg = torch.empty(n, dtype=torch.float64, device="cuda")
            bp = torch.empty_like(bg)
            pgb.pgb_rhs(cg, bg)
            pgb.pgb_rhs(cp, bp)
            assert torch.equal(bg, bp)
    finally:
        pgb.pgb_destroy(cg)
        pgb.pgb_destroy(cp)


@pytest.mark.parametrize("mode", ["fp64", "refine"])
def test_charged_brick_at_zero_ionic_strength(mode):
    """Flat faces, edges and corners in the near field, and kappa = 0 (the
    Yukawa kernels become Laplace's): a sphere molecule over a charged box."""
    v, f = synth.brick(12.0, 12.0, 3.0, 1.5, center=(0.0, 0.0, -8.0))
    bodies = spheres(level_mol=2, surface=False)
    bodies.append(dict(kind="sigma", verts=v, tris=f, eps_in=1.0, qxyz=np.zeros((0, 3)), q=np.zeros(0), bc=0.02))
    so = oracle_system(bodies, kappa=0.0, theta=0.0)
    ctx = gpu_context(bodies, kappa=0.0, theta=0.0)
    try:
        n = pgb.pgb_num_unknowns(ctx)
        x = torch.empty(n, dtype=torch.float64, device="cuda")
        m = pgb.PGB_FP64 if mode == "fp64" else pgb.PGB_FP32_REFINE
        code, st = pgb.pgb_solve(ctx, m, 1e-10, 2000, 100, x)
        assert code == 0
        xo = so.solve()
        assert np.abs(x.cpu().numpy() - xo).max() / np.abs(xo).max() < 1e-8
        e, eo = pgb.pgb_energy(ctx, x), energies(so, xo)
        for k in ("solvation", "surface", "total"):
            assert e[k] == pytest.approx(eo[k], rel=1e-8, abs=1e-12)
    finally:
        pgb.pgb_destroy(ctx)


@pytest.mark.parametrize("mode", ["fp64", "fp32", "refine"])
@pytest.mark.parametrize("precond", [0, 1])
def test_iteration_graph_matches_host_loop(mode, precond):
    """GMRES iterations replayed from the graph with the device-side loop
    (graphs = 2) make the same iterations and the bit-identical solution as
    the host-driven loop (graphs = 0), over restart cycles (restart 8), a
    rebuilt tree (graph recaptured) and a second solve (graph reused)."""
    m = {"fp64": pgb.PGB_FP64, "fp32": pgb.PGB_FP32, "refine": pgb.PGB_FP32_REFINE}[mode]
    tol = 1e-6 if mode == "fp32" else 1e-9
    bodies = spheres(**CASES["sigma_pair"])
    cg = gpu_context(bodies, theta=0.5, P=5, leaf_size=8, graphs=2, precond=precond)
    cp = gpu_context(bodies, theta=0.5, P=5, leaf_size=8, graphs=0, precond=precond)
    try:
        n = pgb.pgb_num_unknowns(cg)
        for step in range(3):
            if step == 1:
                for c in (cg, cp):
                    pgb.pgb_tree_reset(c)
                    pgb.pgb_tree_build(c)
            out = []
            for c in (cg, cp):
                x = torch.empty(n, dtype=torch.float64, device="cuda")
                code, st = pgb.pgb_solve(c, m, tol, 1000, 8, x)
                assert code == 0
                out.append((x.cpu().numpy(), st))
            assert out[0][1]["iterations"] == out[1][1]["iterations"] > 8
            assert out[0][1]["matvecs"] == out[1][1]["matvecs"]
            assert np.array_equal(out[0][0], out[1][0])
    finally:
        pgb.pgb_destroy(cg)
        pgb.pgb_destroy(cp)


@pytest.mark.parametrize("P", [10, 12, 15])
def test_high_order_treecode_matches_oracle_treecode(P):
    """Orders above 8 (Tables 1 and 2 use P = 15): the kernels that stage
    the far coefficients without the register prefetch, the far-field table
    read from L2 with several nodes per block, and the upward pass with its
    children shifted in batches give the oracle treecode's product (same
    lists, same truncated expansion) in FP64, double-single and FP32."""
    bodies = spheres(**CASES["sigma_pair"])
    so = oracle_system(bodies, theta=0.5, P=P, leaf_size=8)
    ctx = gpu_context(bodies, theta=0.5, P=P, leaf_size=8)
    try:
        x = np.random.default_rng(3).normal(size=so.n)
        ref = TreecodeOperator(so).apply(x)
        scale = np.abs(ref).max()
        y64 = _matvec(ctx, x, pgb.PGB_FP64)
        assert np.abs(y64 - ref).max() / scale < 1e-10
        yds = _matvec(ctx, x, pgb.PGB_FP64_DS)
        assert np.abs(yds - y64).max() / scale < 1e-12
        y32 = _matvec(ctx, x, pgb.PGB_FP32)
        assert np.abs(y32 - ref).max() / scale < 2e-5
        # the far field is in use: the product differs from the direct sum
        # by more than round-off, and by less as P grows (Section 3.2)
        direct = so.apply(x)
        assert np.abs(ref - direct).max() / scale > 1e-12
    finally:
        pgb.pgb_destroy(ctx)


def test_orders_without_kernels_are_rejected():
    bodies = spheres(**CASES["sigma_pair"])
    for P in (9, 11, 13, 14, 16):
        with pytest.raises(pgb.PgbError):
            gpu_context(bodies, theta=0.5, P=P)
    ctx = gpu_context(bodies, theta=0.5, P=10)
    try:
        n = pgb.pgb_num_unknowns(ctx)
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        with pytest.raises(pgb.PgbError):
            pgb.pgb_grad(ctx, x, 0, 0, pgb.PGB_FP64, 1e-8, 100, 50)
    finally:
        pgb.pgb_destroy(ctx)


@pytest.mark.parametrize("case", ["sigma_pair", "phi_pair"])
def test_direct_sum_with_37_point_close_by_rule(case):
    """Table 1's close-by rule (37 points, degree 13) in the near-field
    corrections: the direct-sum product matches the oracle's with the same
    rule (each side derives the rule on its own from the moment equations),
    and differs from the 19-point product by the quadrature error."""
    bodies = spheres(**CASES[case])
    so = oracle_system(bodies, theta=0.0, K_near=37)
    ctx = gpu_context(bodies, theta=0.0, leaf_size=16, K_near=37)
    c19 = gpu_context(bodies, theta=0.0, leaf_size=16)
    try:
        x = np.random.default_rng(4).normal(size=so.n)
        ref = so.apply(x)
        scale = np.abs(ref).max()
        y64 = _matvec(ctx, x, pgb.PGB_FP64)
        assert np.abs(y64 - ref).max() / scale < 1e-11
        y32 = _matvec(ctx, x, pgb.PGB_FP32)
        assert np.abs(y32 - ref).max() / scale < 2e-6
        d = np.abs(_matvec(c19, x, pgb.PGB_FP64) - y64).max() / scale
        assert 1e-12 < d < 1e-3
    finally:
        pgb.pgb_destroy(ctx)
        pgb.pgb_destroy(c19)

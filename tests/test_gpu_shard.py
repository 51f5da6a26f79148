"""One solve sharded over two ranks (pgb_matvec_shard, pgb_solve_shard):
two processes on the one GPU with gloo collectives (host-side exchanges; no
kernel waits for another process).  Each rank's rows of the product equal
those rows of the whole product, and the sharded solve gives the energies of
the unsharded one."""
import os
import socket

import numpy as np
import pytest

from problems import gpu_context, spheres

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no GPU", allow_module_level=True)

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import paper_1506_03745_gb300 as pgb  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _bodies():
    return spheres(level_mol=3, level_srf=3, kind="sigma")


def _worker(rank, world, port, q):
    import sys
    sys.path[:0] = [os.path.dirname(os.path.abspath(__file__))]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1506_03745_gb300.shard import solve_sharded
        torch.cuda.set_device(0)
        ctx = gpu_context(_bodies(), theta=0.5, P=6)
        try:
            n = pgb.pgb_num_unknowns(ctx)
            rb = pgb.pgb_shard_rows(ctx, world)
            # this rank's rows of the product against the whole product
            x = torch.tensor(np.random.default_rng(5).normal(size=n), device="cuda")
            y = torch.empty_like(x)
            pgb.pgb_matvec(ctx, x, y, pgb.PGB_FP64)
            xs, ys_full = torch.empty_like(x), torch.empty_like(x)
            pgb.pgb_to_sharded(ctx, x, xs)
            pgb.pgb_to_sharded(ctx, y, ys_full)
            ys = torch.empty(int(rb[rank + 1] - rb[rank]), dtype=torch.float64, device="cuda")
            pgb.pgb_matvec_shard(ctx, rank, world, xs, ys, pgb.PGB_FP64)
            rows_equal = bool(torch.equal(ys, ys_full[int(rb[rank]):int(rb[rank + 1])]))
            out = {}
            for name, mode, tol in (("fp64", pgb.PGB_FP64, 1e-11), ("refine", pgb.PGB_FP32_REFINE, 1e-9)):
                code, xsol, st = solve_sharded(ctx, mode, tol, 2000, 100)
                e = pgb.pgb_energy(ctx, xsol)
                xu = torch.empty_like(xsol)
                cu, su = pgb.pgb_solve(ctx, mode, tol, 2000, 100, xu)
                eu = pgb.pgb_energy(ctx, xu)
                out[name] = (code, cu, st["rel_residual"], e["total"], eu["total"], e["solvation"], eu["solvation"])
            q.put((rank, rows_equal, [int(v) for v in rb], out))
        finally:
            pgb.pgb_destroy(ctx)
    except Exception as exc:  # report, do not hang the parent
        q.put((rank, None, None, repr(exc)))
    finally:
        dist.destroy_process_group()


def test_sharded_solve_over_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = [q.get(timeout=600) for _ in range(2)]
    for p in ps:
        p.join(timeout=120)
    for rank, rows_equal, rb, out in res:
        assert rows_equal is not None, out
        assert rows_equal, rank
        assert rb[0] == 0 and 0 < rb[1] < rb[2]
        for name, (code, cu, rel, e, eu, s, su) in out.items():
            assert code == 0 and cu == 0, name
            assert e == pytest.approx(eu, rel=1e-10 if name == "fp64" else 1e-8), name
            assert s == pytest.approx(su, rel=1e-10 if name == "fp64" else 1e-8), name
    # both ranks hold the same solution
    assert res[0][3]["fp64"][3] == res[1][3]["fp64"][3]

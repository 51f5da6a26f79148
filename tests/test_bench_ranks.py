"""The multi-rank reduction of bench.py (max of the timed intervals, sum of
the work) on two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_max, mv = bench.reduce_across_ranks(dist, 10.0 + 5.0 * rank, 31 + rank, torch.device("cpu"))
    out[rank] = (t_max, mv)
    dist.destroy_process_group()


def test_reduce_across_two_ranks():
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (15.0, 63)


def test_pose_chunks_cover_every_pose_once():
    import bench
    for n, batch in ((4096, 8), (100, 8), (16, 8), (7, 8), (0, 8)):
        for world in (1, 2, 3, 8):
            ranges = [bench.rank_chunks(n, batch, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            for (a, b), (c, d) in zip(ranges, ranges[1:]):
                assert b == c and a <= b
            # whole chunks: every range but the last starts and ends on a chunk boundary
            for a, b in ranges[:-1]:
                assert a % batch == 0 and b % batch == 0
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= batch


def _gather_worker(rank, world, port, out):
    import numpy as np
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    n, batch = 21, 4
    F = np.arange(n * 4, dtype=np.float64).reshape(n, 4) * (rank + 1)  # each rank's copy differs
    lo, hi = bench.rank_chunks(n, batch, rank, world)
    chunks = (n + batch - 1) // batch
    width = ((chunks + world - 1) // world) * batch
    g = bench.gather_rows(dist, F, lo, hi, n, width, torch.device("cpu"))
    out[rank] = None if g is None else g.tolist()
    dist.destroy_process_group()


def test_gather_rows_over_three_ranks():
    import numpy as np
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_gather_worker, args=(3, port, out), nprocs=3, join=True)
    assert out[1] is None and out[2] is None
    import bench
    want = np.zeros((21, 4))
    for r in range(3):
        lo, hi = bench.rank_chunks(21, 4, r, 3)
        want[lo:hi] = (np.arange(84, dtype=np.float64).reshape(21, 4) * (r + 1))[lo:hi]
    assert np.array_equal(np.array(out[0]), want)

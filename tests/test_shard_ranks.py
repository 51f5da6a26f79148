"""Host side of the sharded solve (no GPU): the balanced split of target
groups over ranks (pgb_shard_partition) and the collectives of
paper_1506_03745_gb300.shard over two gloo ranks, on host tensors."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import paper_1506_03745_gb300 as pgb


def test_partition_is_contiguous_and_balanced():
    rng = np.random.default_rng(0)
    work = rng.uniform(1.0, 10.0, size=1000)
    for world in (1, 2, 3, 8):
        b = pgb.pgb_shard_partition(work, world)
        assert b[0] == 0 and b[-1] == len(work)
        assert np.all(np.diff(b) >= 1)
        tot = work.sum()
        shares = np.array([work[b[r]:b[r + 1]].sum() for r in range(world)])
        # each boundary sits within one group of the ideal split
        assert np.all(np.abs(shares - tot / world) <= work.max() + 1e-9)


def test_partition_edge_cases():
    # fewer groups than ranks: contiguous, non-decreasing, all groups covered
    b = pgb.pgb_shard_partition(np.ones(3), 5)
    assert b[0] == 0 and b[-1] == 3 and np.all(np.diff(b) >= 0)
    assert list(pgb.pgb_shard_partition(np.zeros(0), 2)) == [0, 0, 0]
    assert list(pgb.pgb_shard_partition(np.ones(4), 1)) == [0, 4]
    with pytest.raises(pgb.PgbError):
        pgb.pgb_shard_partition(np.array([1.0, -1.0]), 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, rows, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1506_03745_gb300.shard import Collectives
        rb = np.concatenate([[0], np.cumsum(rows)])
        n = int(rb[-1])
        xs = torch.full((n,), -1.0, dtype=torch.float64)
        xs[rb[rank]:rb[rank + 1]] = torch.arange(rb[rank], rb[rank + 1], dtype=torch.float64) * 10 + rank
        red = torch.tensor([1.0 + rank, 2.0 * rank, 5.0, 7.0], dtype=torch.float64)
        c = Collectives(xs, red, rb)
        assert c(None, 0, n) == 0           # allgather
        assert c(None, 1, 3) == 0           # allreduce of the first three
        q.put((rank, xs.numpy().copy(), red.numpy().copy()))
    finally:
        dist.destroy_process_group()


def test_collectives_over_two_gloo_ranks():
    """Uneven row ranges gathered on both ranks; the first three entries of
    the reduce buffer summed, the fourth left alone."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    rows = [5, 3]
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, rows, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = np.array([i * 10 + (0 if i < 5 else 1) for i in range(8)], dtype=float)
    for rank, xs, red in out:
        np.testing.assert_array_equal(xs, want)
        np.testing.assert_array_equal(red[:3], [1.0 + 2.0, 0.0 + 2.0, 10.0])
        assert red[3] == 7.0

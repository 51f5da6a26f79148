"""One solve sharded over ranks (pgb_solve_shard): the collectives the
library asks for, done with torch.distributed (NCCL between GPUs, gloo
between CPU ranks).  Argument marshalling and transport only: the products,
the Arnoldi arithmetic and the refinement run in the library.

    import torch.distributed as dist
    dist.init_process_group("nccl")          # or "gloo"; one rank per GPU
    x, stats = solve_sharded(ctx, PGB_FP32_REFINE, 1e-6)
"""
import ctypes

import numpy as np
import torch
import torch.distributed as dist

from . import _lib as L

_CB = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64)


class Collectives:
    """The allgather of a rank's rows of the exchange vector xs (sharded order,
    rows row_begin[r] .. row_begin[r + 1] per rank) and the allreduce of the
    first count entries of red, over a torch.distributed process group.  With
    the gloo backend the tensors pass through host memory."""

    def __init__(self, xs, red, row_begin, group=None):
        self.xs, self.red = xs, red
        self.rb = [int(v) for v in row_begin]
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.host = dist.get_backend(group) == "gloo"
        self.rows = max(self.rb[r + 1] - self.rb[r] for r in range(self.world))
        self.error = None

    def _sync(self):
        if self.xs.is_cuda:
            torch.cuda.synchronize(self.xs.device)

    def allgather(self):
        lo, hi = self.rb[self.rank], self.rb[self.rank + 1]
        dev = torch.device("cpu") if self.host else self.xs.device
        send = torch.zeros(self.rows, dtype=self.xs.dtype, device=dev)  # equal sizes for all_gather
        send[:hi - lo].copy_(self.xs[lo:hi])
        recv = [torch.empty_like(send) for _ in range(self.world)]
        dist.all_gather(recv, send, group=self.group)
        for r in range(self.world):
            a, b = self.rb[r], self.rb[r + 1]
            if r != self.rank:
                self.xs[a:b].copy_(recv[r][:b - a])
        self._sync()

    def allreduce(self, count):
        t = self.red[:count].cpu() if self.host else self.red[:count]
        dist.all_reduce(t, group=self.group)
        if self.host:
            self.red[:count].copy_(t)
        self._sync()

    def __call__(self, user, op, count):
        try:
            if op == L.PGB_COLL_ALLGATHER:
                self.allgather()
            elif op == L.PGB_COLL_ALLREDUCE:
                self.allreduce(int(count))
            else:
                return 1
            return 0
        except Exception as e:  # reported as PGB_ECOLL by the library
            self.error = e
            return 1


def shard_rows(ctx, world):
    return L.pgb_shard_rows(ctx, world)


def solve_sharded(ctx, mode, tol, max_iter=2000, restart=100, group=None):
    """Sharded solve on this rank of `group` (every rank calls it with the
    same context contents): returns (status, solution x in the caller's order
    on this rank's device, stats dict)."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    n = L.pgb_num_unknowns(ctx)
    rb = L.pgb_shard_rows(ctx, world)
    dev = torch.device("cuda", torch.cuda.current_device())
    xs = torch.zeros(n, dtype=torch.float64, device=dev)
    red = torch.zeros(restart + 2, dtype=torch.float64, device=dev)
    coll = Collectives(xs, red, rb, group)
    cb = _CB(coll)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    code, st = L.pgb_solve_shard(ctx, rank, world, xs, red, cb, mode, tol, max_iter, restart, x)
    if coll.error is not None:
        raise coll.error
    return code, x, st

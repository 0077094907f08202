"""Multi-rank GRPIC step: particles sharded over ranks, the grid replicated.

Every rank pushes and deposits its own particles; the deposit's outputs (rho
and the three currents, each already divided by its node volume, so partial
sums add) are summed over the ranks before the field update, which every
rank then runs on identical sources, keeping the replicated fields identical.
The sum is the step's one exchange (Sec. 2.1: the currents couple the
particles to Maxwell's equations); on GPUs it runs through NCCL, in the tests
through gloo on CPU.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def sharded() -> bool:
    """True when the step runs on more than one rank."""
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def allreduce_sources(tensors, group=None) -> None:
    """Sum the deposit's rho, J^r, J^th, J^ph over the ranks, in place."""
    if not sharded():
        return
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)


def shard_bounds(n: int, rank: int, world: int) -> tuple[int, int]:
    """[begin, end) of rank's share of n particles (contiguous, balanced)."""
    return n * rank // world, n * (rank + 1) // world


def assert_replicas_equal(tensors, group=None) -> None:
    """Check that a replicated array is bitwise the same on every rank."""
    if not sharded():
        return
    for t in tensors:
        ref = t.clone()
        dist.broadcast(ref, src=0, group=group)
        if not torch.equal(ref, t):
            raise RuntimeError("replicated field arrays differ between ranks")

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


def _flat_span(tensors):
    """One 1-D view covering every tensor when they are equally strided
    slices of one storage laid out in order (fpic.Fields keeps a level's
    rho, J^r, J^th, J^ph that way), else None."""
    t0 = tensors[0]
    if any(t.dtype != t0.dtype or t.device != t0.device or not t.is_contiguous() or t.dim() != 1 for t in tensors):
        return None
    st = t0.untyped_storage()
    if any(t.untyped_storage().data_ptr() != st.data_ptr() for t in tensors):
        return None
    offs = [t.storage_offset() for t in tensors]
    step = offs[1] - offs[0] if len(offs) > 1 else t0.numel()
    if step < t0.numel() or any(offs[k] != offs[0] + k * step for k in range(len(offs))) or \
            any(t.numel() != t0.numel() for t in tensors):
        return None
    flat = torch.empty(0, dtype=t0.dtype, device=t0.device)
    return flat.set_(st, offs[0], (step * (len(tensors) - 1) + t0.numel(),))


def allreduce_sources(tensors, group=None) -> None:
    """Sum the deposit's rho, J^r, J^th, J^ph over the ranks, in place, with
    one all-reduce: over the buffer the four arrays share when they are
    slices of one (fpic.Fields), else over a packed copy."""
    if not sharded():
        return
    flat = _flat_span(tensors)
    if flat is not None:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
        return
    packed = torch.cat([t.reshape(-1) for t in tensors])
    dist.all_reduce(packed, op=dist.ReduceOp.SUM, group=group)
    o = 0
    for t in tensors:
        t.copy_(packed[o:o + t.numel()].view_as(t))
        o += t.numel()


def assign_runs(counts, world: int):
    """Independent runs of a batch (split-monopole workload: one run per
    spacetime) over `world` ranks, balancing particles: runs taken largest
    first, each to the rank with the fewest particles so far (ties: the
    lower rank).  Returns, per rank, the sorted list of its run indices.
    No exchange follows: each rank pushes its runs as one batch of its own."""
    load = [0] * world
    out = [[] for _ in range(world)]
    for i in sorted(range(len(counts)), key=lambda i: (-counts[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += counts[i]
    return [sorted(x) for x in out]


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

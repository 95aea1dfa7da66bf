"""Sharding across ranks: contiguous segment ranges with global segment ids
(the counter-based draws make any partition give the same photons) and an
exact reduction of the integer outputs.  One process per GPU; the reduce uses
torch.distributed (NCCL on GPUs, gloo on CPU ranks)."""
from __future__ import annotations


def shard_range(n: int, rank: int, world: int):
    """[start, stop) of rank's contiguous share of n segments; start is also
    the shard's seg_base (its first global segment id)."""
    if not (0 <= rank < world):
        raise ValueError("rank %d outside world %d" % (rank, world))
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def reduce_counts(tensors, group=None, dst=None):
    """Sums output tensors over the ranks in place (all_reduce, or reduce to
    dst).  Integer sums are exact, so the combined histogram, telescope counts
    and counters equal the single-process ones bit for bit.  The float64
    arrival-time sums are not: the order in which the ranks' partial sums are
    added is the collective's, so they agree with one process to a relative
    1e-12 (each sum holds at most a few thousand terms of similar size)."""
    import torch
    import torch.distributed as dist
    for t in tensors:
        if t.dtype not in (torch.int64, torch.int32, torch.float64):
            raise TypeError("reduce_counts expects int64/int32 counts or float64 time sums")
        if dst is None:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        else:
            dist.reduce(t, dst=dst, op=dist.ReduceOp.SUM, group=group)
    return tensors

"""Splitting the stacks of a workload over processes (one per GPU).

Stacks are independent (Sec. II: each is its own 1-D problem), so a workload
shards by stack with no exchange on the data path: rank r runs a contiguous
range of stacks in its own context, with `stack_base` set to the global
index of its first stack so that every stack draws the same random streams
as in a single context.  The only collective is the reduction of the timing
and the counts at the end of a measurement.
"""
from __future__ import annotations


def stack_range(weights, rank: int, world: int):
    """Contiguous [lo, hi) of the stacks for `rank`, balanced by weight (the
    carriers a stack starts with); every stack belongs to exactly one rank."""
    n = len(weights)
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d of %d" % (rank, world))
    total = float(sum(weights))
    bounds, acc, j = [0], 0.0, 0
    for r in range(1, world):
        target = total * r / world
        while j < n and acc + weights[j] / 2.0 <= target:
            acc += weights[j]
            j += 1
        bounds.append(max(j, bounds[-1]))
    bounds.append(n)
    return bounds[rank], bounds[rank + 1]


def shard(wl, rank: int, world: int):
    """The workload of `rank`: (its stacks as a workload, stack_base)."""
    lo, hi = stack_range([st.n0 for st in wl.stacks], rank, world)
    return wl.replace(stacks=list(wl.stacks[lo:hi])), lo


def reduce_measurement(ms: float, count: float, dist=None, device=None):
    """Whole-job figures of a timed region: the largest time over the ranks
    and the sum of the units (carrier-steps) they processed."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, count
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    c = torch.tensor([count], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())

"""Problem sharding across ranks (one process per GPU).

Independent point-source problems (sources, frequencies) need no exchange: each
rank solves its own share.  The collectives are the timing reduction (max
over ranks) that reports the whole job's time and, for the receiver-misfit
gradient, one all-reduce sum of the per-rank misfit and slowness gradient
(`sharded_sum`).  A single solve is not split across GPUs (it would need a
halo exchange per stencil apply and an all-reduce per Krylov dot).
"""
from __future__ import annotations

import os


def env():
    """(rank, world_size, local_rank) from the torch.distributed launcher's environment."""
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def partition(count, rank, world, weights=None):
    """Indices of the problems rank `rank` of `world` solves.

    Without weights: a contiguous, near-equal split (the first count % world
    ranks take one more).  With weights (e.g. nodes x expected iterations per
    problem): greedy longest-processing-time assignment, deterministic (ties by
    index), so every rank computes the same assignment without communication.
    """
    if world < 1 or not (0 <= rank < world):
        raise ValueError("rank must be in [0, world)")
    if weights is None:
        base, extra = divmod(count, world)
        lo = rank * base + min(rank, extra)
        hi = lo + base + (1 if rank < extra else 0)
        return list(range(lo, hi))
    if len(weights) != count:
        raise ValueError("one weight per problem")
    load = [0.0] * world
    owner = [0] * count
    for i in sorted(range(count), key=lambda k: (-weights[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += weights[i]
    return [i for i in range(count) if owner[i] == rank]


def max_over_ranks(value, device=None):
    """The maximum of a float over all ranks (the value itself on one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, device=None):
    """The sum of a number over all ranks (problem counts)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.item()


def sharded_sum(count, per_item, rank=None, world=None, weights=None, out=None):
    """Sum of per_item(i) -> (scalar, tensor) over i in [0, count), each rank
    evaluating its `partition` share, then one all-reduce sum over the ranks.

    The gradient of a multi-source misfit is a sum over sources, so ranks
    that solve disjoint sources only exchange their partial sums once, at the
    end: the scalar rides in the last entry of one all-reduce buffer with the
    tensor.  rank / world default to the initialised process group (else 0
    and 1); `out` (a tensor shaped like per_item's) receives this rank's sum
    before the reduction, and the total after it.  Returns (scalar, tensor).
    """
    import torch
    import torch.distributed as dist
    grouped = dist.is_available() and dist.is_initialized()
    if rank is None or world is None:
        rank, world = (dist.get_rank(), dist.get_world_size()) if grouped else (0, 1)
    mine = partition(count, rank, world, weights)
    scalar, total = 0.0, out
    for i in mine:
        s, t = per_item(i)
        scalar += float(s)
        if total is None:
            total = t.clone()
        elif t is not total:
            total += t
    if total is None:
        raise ValueError("no item on this rank and no `out` tensor to shape the reduction")
    if world == 1 or not grouped:
        return scalar, total
    buf = torch.cat([total.reshape(-1).to(torch.float64), torch.tensor([scalar], dtype=torch.float64,
                                                                        device=total.device)])
    dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    total.copy_(buf[:-1].reshape(total.shape).to(total.dtype))
    return float(buf[-1].item()), total

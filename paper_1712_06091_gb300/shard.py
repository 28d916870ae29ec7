"""Problem sharding across ranks (one process per GPU).

Independent point-source problems (sources, frequencies) need no exchange: each
rank solves its own share, and the only collective is the timing reduction
(max over ranks) that reports the whole job's time.  A single solve is not
split across GPUs (it would need a halo exchange per stencil apply and an
all-reduce per Krylov dot).
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

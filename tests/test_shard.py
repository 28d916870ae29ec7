"""Multi-rank host logic on CPU (gloo, world size 2): problem partitions cover
every problem exactly once with no communication, and the timing reduction
takes the slowest rank."""
import os
import socket

import pytest

from paper_1712_06091_gb300 import shard


@pytest.mark.parametrize("count,world", [(96, 2), (7, 3), (3, 4), (0, 2)])
def test_partition_covers_each_problem_once(count, world):
    parts = [shard.partition(count, r, world) for r in range(world)]
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(count))
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1


def test_weighted_partition_balances_load():
    weights = [65 ** 3] * 32 + [97 ** 3] * 32 + [129 ** 3] * 32
    parts = [shard.partition(len(weights), r, 2, weights) for r in range(2)]
    assert sorted(i for p in parts for i in p) == list(range(96))
    loads = [sum(weights[i] for i in p) for p in parts]
    assert abs(loads[0] - loads[1]) <= max(weights)
    assert parts == [shard.partition(len(weights), r, 2, weights) for r in range(2)]   # deterministic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, _ = shard.env()
        mine = shard.partition(10, r, w)
        slowest = shard.max_over_ranks(1.5 + r)          # rank 1 is slower
        total = shard.sum_over_ranks(len(mine))
        out.put((r, mine, slowest, total))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sharding():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    results = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [r[1] for r in results] == [[0, 1, 2, 3, 4], [5, 6, 7, 8, 9]]
    assert all(r[2] == 2.5 for r in results)
    assert all(r[3] == 10 for r in results)


def _item(i, n=64):
    """A source's misfit and gradient stand-in: deterministic per index."""
    import torch
    g = torch.Generator().manual_seed(1000 + i)
    return float(i * i + 0.5), torch.randn(n, dtype=torch.float64, generator=g)


def _gradient_worker(rank, world, port, count, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seen = []

        def accumulate(i, acc=torch.zeros(64, dtype=torch.float64)):
            # the misfit_gradient pattern: every source adds into one buffer
            seen.append(i)
            J, g = _item(i)
            acc += g
            return J, acc

        buf = torch.zeros(64, dtype=torch.float64)
        J, grad = shard.sharded_sum(count, lambda i: accumulate(i, buf), out=buf)
        out.put((rank, seen, J, grad.numpy().tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("count,world", [(16, 2), (2, 3)])
def test_sharded_gradient_allreduce_gloo(count, world):
    """The sharded misfit gradient: each rank sums its partition's sources and
    one all-reduce gives every rank the single-rank total (a rank without a
    source contributes zeros)."""
    import numpy as np
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gradient_worker, args=(r, world, port, count, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted((out.get(timeout=120) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(i for r in results for i in r[1]) == list(range(count))   # every source once
    J_ref = sum(_item(i)[0] for i in range(count))
    g_ref = sum(_item(i)[1].numpy() for i in range(count))
    for _, _, J, g in results:
        assert abs(J - J_ref) <= 1e-12 * J_ref
        assert np.allclose(np.array(g), g_ref, rtol=1e-13, atol=1e-13)


def test_sharded_sum_single_process():
    import torch
    J, g = shard.sharded_sum(5, _item, rank=0, world=1)
    assert abs(J - sum(_item(i)[0] for i in range(5))) < 1e-12
    assert torch.allclose(g, sum(_item(i)[1] for i in range(5)))

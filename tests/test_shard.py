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

"""Multi-rank host logic on CPU: domain sharding and the max-over-ranks timing reduction, run as
two gloo ranks (the GPU path itself runs one process per GPU with no data-path collective)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2609_30039_gb300 import sharding
from paper_2609_30039_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_shard_domains_partition_and_balance():
    scs = W.lorentz_batch()
    cells = [sc.cells for sc in scs]
    for world in (1, 2, 3, 4, 8):
        shards = sharding.shard_domains(cells, world)
        flat = sorted(d for s in shards for d in s)
        assert flat == list(range(len(cells)))          # every domain exactly once
        loads = [sum(cells[d] for d in s) for s in shards]
        assert max(loads) - sum(loads) / world < max(cells)   # LPT bound
        assert shards == sharding.shard_domains(cells, world)  # deterministic


def test_shard_domains_more_ranks_than_domains():
    shards = sharding.shard_domains([10, 20], 4)
    assert sorted(d for s in shards for d in s) == [0, 1]
    assert sum(1 for s in shards if not s) == 2
    with pytest.raises(ValueError):
        sharding.shard_domains([1], 0)


def _rank_main(rank, world, port, cells, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = sharding.shard_domains(cells, world)[rank]
        t_ms = 10.0 + 5.0 * rank                      # this rank's "measured" time
        t_max = sharding.max_over_ranks(t_ms, dist)
        n = sharding.sum_over_ranks(sum(cells[d] for d in mine), dist)
        got = [None] * world
        dist.all_gather_object(got, mine)
        q.put((rank, t_max, n, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    cells = [sc.cells for sc in W.lorentz_batch()]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, cells, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, n, got in res:
        assert t_max == 15.0                            # the slowest rank's time on every rank
        assert n == sum(cells)                          # all cells advanced exactly once
        assert sorted(d for s in got for d in s) == list(range(len(cells)))
        assert got == sharding.shard_domains(cells, world)


def test_single_process_reductions_are_identity():
    assert sharding.max_over_ranks(3.5) == 3.5
    assert sharding.sum_over_ranks(7) == 7.0

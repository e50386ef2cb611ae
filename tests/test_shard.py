"""Placement of independent problems on ranks: the partition covers every
problem once, balances the work estimate, and agrees across ranks; the
max-over-ranks reduction of the benchmark works over a world_size-2 gloo
group (CPU)."""
import os
import socket

import pytest

from paper_2105_01722_gb300 import inputs, shard


def test_partition_covers_disjoint_and_balanced():
    specs = inputs.batched_problems(48)
    for world in (1, 2, 3, 4, 8):
        parts = shard.partition(specs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(specs)))
        loads = [sum(shard.work_estimate(specs[i]) for i in p) for p in parts]
        biggest = max(shard.work_estimate(s) for s in specs)
        # greedy LPT: no rank exceeds the mean by more than the largest item
        assert max(loads) <= sum(loads) / world + biggest + 1e-9


def test_partition_is_deterministic_and_rejects_bad_world():
    specs = inputs.batched_problems(20)
    assert shard.partition(specs, 3) == shard.partition(list(specs), 3)
    with pytest.raises(ValueError):
        shard.partition(specs, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        specs = inputs.batched_problems(48)
        mine = shard.partition(specs, world)[rank]
        # every rank computes the same placement: gather and compare
        objs = [None] * world
        dist.all_gather_object(objs, shard.partition(specs, world))
        same = all(o == objs[0] for o in objs)
        t = shard.max_over_ranks(1.5 + rank)
        q.put((rank, mine, same, t))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert all(r[2] for r in res)
    assert all(r[3] == 2.5 for r in res)                 # max over ranks
    assert sorted(res[0][1] + res[1][1]) == list(range(48))
    assert not set(res[0][1]) & set(res[1][1])

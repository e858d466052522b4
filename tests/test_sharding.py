"""Host logic of the multi-GPU path on CPU: instance sharding and the max-over-ranks
time, with two gloo ranks (no GPU)."""
import os
import socket

import pytest

from paper_2412_18829_gb300 import sharding
import synth


def test_shard_is_a_partition_and_balanced():
    sizes = [int(n) for n in synth.batch_c4_sizes()]
    costs = [sharding.build_cost(n, 6 * n, 120) for n in sizes]
    for world in (1, 2, 3, 4, 8, 16, 20):
        parts = sharding.shard(costs, world)
        assert len(parts) == world
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        if world <= len(costs):
            loads = [sum(costs[i] for i in p) for p in parts]
            # LPT bound: the busiest rank holds at most the mean plus the largest item
            assert max(loads) <= sum(costs) / world + max(costs) + 1e-6


def test_shard_rejects_empty_world():
    with pytest.raises(ValueError):
        sharding.shard([1.0], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = [int(n) for n in synth.batch_c4_sizes()]
        mine = sharding.shard([sharding.build_cost(n, 6 * n, 120) for n in sizes], world)[rank]
        got = [None] * world
        dist.all_gather_object(got, mine)
        t = sharding.max_over_ranks(0.5 + rank, dist)
        q.put((rank, got, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_partition_and_the_slowest_time():
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
    for rank, got, t in res:
        assert sorted(i for part in got for i in part) == list(range(16))
        assert got[rank] == sharding.shard([sharding.build_cost(int(n), 6 * int(n), 120)
                                            for n in synth.batch_c4_sizes()], 2)[rank]
        assert t == 1.5

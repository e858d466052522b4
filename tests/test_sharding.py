"""Host logic of the multi-GPU path on CPU: instance sharding and the max-over-ranks
time, with two gloo ranks (no GPU)."""
import os
import socket

import numpy as np
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


@pytest.mark.parametrize("n_tau", [2, 3, 8, 30, 31, 80])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_tau_shards_partition_the_grid_in_mirror_pairs(n_tau, world):
    if world > n_tau // 2:   # some rank would get no mirror pair: refused up front
        with pytest.raises(ValueError):
            sharding.tau_shards(n_tau, world)
        return
    parts = sharding.tau_shards(n_tau, world)
    assert sorted(j for p in parts for j in p) == list(range(n_tau))
    for p in parts:
        assert sharding.compact_is_mirror(p, n_tau)
        assert len(p) >= 2   # every shard is a grid sox_sigma accepts (n_tau >= 2)
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 3


def test_compact_grid_reproduces_the_full_build():
    """Sigma on each rank's compact G equals the full build's slices (oracle, CPU)."""
    from oracle import sox

    w = synth.tiny(4, 9, n_tau=7)
    full = sox.sox_sigma(w.X, w.V, w.G)
    parts, orders = [], sharding.tau_shards(w.n_tau, 3)
    for order in orders:
        parts.append(sox.sox_sigma(w.X, w.V, w.G[:, :, order]))
    got = sharding.assemble(parts, orders, w.n_tau)
    assert np.abs(got - full).max() <= 1e-15 * np.abs(full).max()


def _tau_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from oracle import sox

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.tiny(3, 7, n_tau=6)
        orders = sharding.tau_shards(w.n_tau, world)
        mine = torch.from_numpy(sox.sox_sigma(w.X, w.V, w.G[:, :, orders[rank]]).real.copy())
        got = [None] * world
        dist.all_gather_object(got, mine)
        full = sharding.assemble(got, orders, w.n_tau)
        ref = sox.sox_sigma(w.X, w.V, w.G).real
        q.put((rank, float(np.abs(full.numpy() - ref).max()), float(np.abs(ref).max())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_one_build_by_tau():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_tau_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, err, scale in res:
        assert err <= 1e-15 * scale


@pytest.mark.parametrize("n,world", [(1, 1), (5, 2), (7, 3), (120, 8), (26, 4)])
def test_v_shards_partition_the_orbital_index(n, world):
    parts = sharding.v_shards(n, world)
    assert len(parts) == world
    assert parts[0][0] == 0 and parts[-1][1] == n
    for (a, b), (c, _) in zip(parts, parts[1:]):
        assert b == c
    sizes = [b - a for a, b in parts]
    assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1


def test_v_shards_refuse_more_ranks_than_orbitals():
    with pytest.raises(ValueError):
        sharding.v_shards(3, 4)
    with pytest.raises(ValueError):
        sharding.v_shards(3, 0)


def _mask_columns(Gm, v0, v1):
    """G(-tau) with the columns v outside [v0, v1) set to zero: Eq. (sox) then keeps only the
    terms of the rank's v range (v enters through G_sv(-tau) and the mixed tensor U2_Rvw,
    whose products with the zeroed columns vanish)."""
    out = np.zeros_like(Gm)
    out[..., v0:v1] = Gm[..., v0:v1]
    return out


def _v_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    from oracle import grid, kpoints, sox

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        # molecule: partial Sigma of the rank's v range at every tau, summed over ranks
        w = synth.tiny(5, 11, n_tau=4)
        v0, v1 = sharding.v_shards(w.n, world)[rank]
        Gm = grid.g_minus_tau(w.G[0, 0].astype(complex))
        part = np.stack([sox.sigma_chain(w.X[0], w.V[0], w.V[0], w.G[0, 0, j], _mask_columns(Gm[j], v0, v1))
                         for j in range(w.n_tau)])
        t = torch.from_numpy(np.ascontiguousarray(part.real))
        dist.all_reduce(t)
        full = sox.sox_sigma(w.X, w.V, w.G)[0, 0].real
        out["molecule"] = (float(np.abs(t.numpy() - full).max()), float(np.abs(full).max()))
        # solid: the momentum-resolved chain, G(-tau)^k masked for every k
        s = synth.solid(9, (1, 1, 2), 4, 9, 3, 10.0)
        v0, v1 = sharding.v_shards(s.n, world)[rank]
        Gs = np.asarray(s.G[0], complex)
        Gms = grid.g_minus_tau(Gs)
        part = np.stack([kpoints.sigma_chain(s.X, s.V, s.V, Gs[:, j], _mask_columns(Gms[:, j], v0, v1), s.nk)
                         for j in range(s.n_tau)])
        t = torch.from_numpy(np.ascontiguousarray(part))
        dist.all_reduce(t)
        full = kpoints.sox_sigma(s.X, s.V, s.G, s.nk)[0].transpose(1, 0, 2, 3)
        out["solid"] = (float(np.abs(t.numpy() - full).max()), float(np.abs(full).max()))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_one_build_by_v():
    """Each rank keeps the terms of its own v range; one all-reduce of the orbital-basis
    Sigma gives the whole build (molecule and solid, oracle chains on CPU)."""
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_v_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, out in res:
        for what, (err, scale) in out.items():
            assert scale > 0
            assert err <= 1e-14 * scale, what

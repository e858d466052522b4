"""Host-side partition of independent SOX problems over ranks (one process per GPU).

The uneven batch of molecules is a set of independent builds: each instance's
Sigma depends on its own G, X and V only (Sec. II C, per instance), so ranks
share no data and need no collective on the data path.  Instances are dealt out
by longest-processing-time first on the algorithmic cost of the fused B/C/D step
(4 N^2 n^2 per tau point and spin), which dominates every build.
"""
from __future__ import annotations


def build_cost(n: int, N: int, n_tau: int, n_spin: int = 1) -> float:
    """Algorithmic flops of the B/C/Hadamard step of one build (2 per multiply-add)."""
    return 4.0 * N * N * n * n * n_tau * n_spin


def shard(costs, world: int) -> list[list[int]]:
    """Indices of `costs` per rank, largest first onto the least-loaded rank.

    Deterministic (ties broken by index and rank), every index appears exactly
    once, and the result is the same on every rank.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += float(costs[i])
    return [sorted(x) for x in out]


def max_over_ranks(t_local: float, dist=None, device=None) -> float:
    """Slowest rank's time: the whole job ends when the last rank does."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(t_local)
    import torch

    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

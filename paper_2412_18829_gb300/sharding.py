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


# ---------------------------------------------------------------------------
# One build split over ranks by tau.  The static chain is local in tau except for the
# reflection G(-tau_j) = -G(tau_{n_tau-1-j}) (Sec. II C on a mirror-symmetric grid), so a
# rank owns whole mirror pairs {j, n_tau-1-j}: packed as [a_1 .. a_k, (mid), mirrors of
# a_k .. a_1], its G slices are themselves mirror-symmetric and sox_sigma on them returns
# exactly the Sigma(tau) of those points.  Gathering the slices is the one exchange.
# ---------------------------------------------------------------------------
def tau_shards(n_tau: int, world: int) -> list[list[int]]:
    """Tau indices per rank in compact (mirror-symmetric) order; every index exactly once.

    The n_tau // 2 mirror pairs are dealt round-robin (equal cost per pair); an odd grid's
    middle point joins the rank with the fewest pairs.  Every shard is itself a valid
    grid for sox_sigma (at least one pair, so at least 2 points): a split with more
    ranks than mirror pairs is refused with ValueError."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if n_tau < 2:
        raise ValueError("n_tau must be >= 2")
    if world > n_tau // 2:
        raise ValueError(f"{n_tau} tau points have {n_tau // 2} mirror pairs: too few for {world} ranks "
                         "(every rank needs a pair)")
    pairs = [[] for _ in range(world)]
    for j in range(n_tau // 2):
        pairs[j % world].append(j)
    mid_rank = min(range(world), key=lambda r: (len(pairs[r]), r)) if n_tau % 2 else None
    out = []
    for r in range(world):
        first = sorted(pairs[r])
        mids = [n_tau // 2] if r == mid_rank else []
        out.append(first + mids + [n_tau - 1 - j for j in reversed(first)])
    return out


def compact_is_mirror(order: list[int], n_tau: int) -> bool:
    """True when position p and len-1-p hold reflected tau indices for every p."""
    m = len(order)
    return all(order[p] + order[m - 1 - p] == n_tau - 1 for p in range(m))


def assemble(parts, orders, n_tau: int, axis: int = 2):
    """Sigma over the full grid from the ranks' compact slices (numpy or torch, along `axis`)."""
    first = parts[0]
    shape = list(first.shape)
    shape[axis] = n_tau
    if hasattr(first, "new_empty"):
        out = first.new_empty(shape)
    else:
        import numpy as np

        out = np.empty(shape, dtype=first.dtype)
    for part, order in zip(parts, orders):
        for p, j in enumerate(order):
            idx = [slice(None)] * len(shape)
            src = [slice(None)] * len(shape)
            idx[axis] = j
            src[axis] = p
            out[tuple(idx)] = part[tuple(src)]
    return out


# ---------------------------------------------------------------------------
# One build split over ranks by the orbital index v.  Eq. (sox) sums over v, the column of
# G(-tau) in G_sv(-tau) (the index the dynamic algorithm of Sec. II C moves to the outside
# loop); every step of the static and dynamic chains is linear in that sum, so a rank that
# keeps only its own v range (sox_set_v_range) returns a partial Sigma, and the sum of the
# partials over a partition of [0, n) is the whole build: one all-reduce of the orbital-basis
# Sigma.  Every v costs the same (one B_v / C_v pair per tile and tau), so equal contiguous
# ranges balance the ranks.  This split also keeps a solid's n_k^3 D step whole: each rank
# runs the Fourier form of the D step over the full k mesh for its own v.
# ---------------------------------------------------------------------------
def v_shards(n: int, world: int) -> list[tuple[int, int]]:
    """Contiguous [v0, v1) ranges of the orbital index, one per rank, sizes differing by at
    most one; every v in exactly one range.  Refuses more ranks than orbitals."""
    if world < 1:
        raise ValueError("world must be >= 1")
    if n < world:
        raise ValueError(f"{n} orbitals cannot give each of {world} ranks a v")
    base, extra = divmod(n, world)
    out, v0 = [], 0
    for r in range(world):
        v1 = v0 + base + (1 if r < extra else 0)
        out.append((v0, v1))
        v0 = v1
    return out


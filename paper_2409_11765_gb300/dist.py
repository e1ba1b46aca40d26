"""Multi-GPU layout of the batched engine: one process per GPU, independent
searches per rank, no collective on the data path.

The paper's K-Distributed strategy (§3.2.3) runs the descents of every
population level at the same time on disjoint groups of processes. On GPUs the
unit of independence is the search: each rank owns whole searches, and the
only communication is
  * the timing barrier and the maximum of the per-rank times,
  * a final gather of every search's (f_best, x_best) to rank 0, and
  * an optional global stop flag: the minimum of f_best over all ranks,
    compared with the target every few generations.
Searches are assigned to ranks by their cost per generation: sampling and
objective work lambda n^2 plus the eigendecomposition n^3 amortised over the
lazy cadence g_eig (the O(lambda n^2) and O(n^3) terms of §2.1).
"""
import math
import os

SEED_STRIDE = 7919


def env():
    """(rank, local_rank, world_size) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def rank_seed(base, rank):
    """Philox key of a rank: distinct streams for every rank's searches."""
    return (int(base) + SEED_STRIDE * int(rank)) & 0xFFFFFFFFFFFFFFFF


def shard(count, world, rank):
    """Contiguous share [lo, hi) of `count` searches for `rank` (sizes differ by
    at most one; every search belongs to exactly one rank)."""
    base, extra = divmod(count, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def lazy_eig_interval(n, lam):
    """Generations between eigendecompositions under the lazy rule
    max(1, floor(1 / ((c1 + c_mu) n 10))), with the default learning rates of
    a descent of size lam (log weights on the best floor(lam/2) points)."""
    mu = lam // 2
    wp = [math.log((lam + 1) / 2.0) - math.log(i) for i in range(1, mu + 1)]
    s1 = sum(wp)
    mueff = s1 * s1 / sum(w * w for w in wp)
    c1 = 2.0 / ((n + 1.3) ** 2 + mueff)
    cmu = min(1.0 - c1, 2.0 * (mueff - 2.0 + 1.0 / mueff) / ((n + 2.0) ** 2 + mueff))
    return max(1, int(math.floor(1.0 / ((c1 + cmu) * n * 10.0))))


def search_cost(n, lam):
    """Work of one generation of one search: lambda n^2 (sampling, objective,
    rank-mu update) plus n^3 / g_eig (the amortised eigendecomposition)."""
    return float(lam) * n * n + float(n) ** 3 / lazy_eig_interval(n, lam)


def assign(costs, world):
    """Whole searches to ranks, balancing the summed cost: longest first, each
    to the least-loaded rank (ties to the lower rank). Returns one ascending
    list of search ids per rank; every search belongs to exactly one rank."""
    load = [0.0] * world
    owned = [[] for _ in range(world)]
    for s in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += costs[s]
        owned[r].append(s)
    return [sorted(o) for o in owned]


def max_over_ranks(value, dist=None, device=None):
    """Largest value over all ranks (the timing rule: the slowest rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def global_min(value, dist=None, device=None):
    """Smallest value over all ranks (the best f of the whole job)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return float(t.item())


def stop_flag(local_best_f, f_target, dist=None, device=None):
    """True on every rank once some rank's best f is below the target: the
    optional global stop, checked every few generations between steps."""
    return global_min(local_best_f, dist, device) < f_target


def gather_best(local, count, dist=None):
    """Every search's (f_best, x_best) on rank 0.

    local: {search id: (f_best, x_best as a sequence of floats)} for the
    searches this rank owns. Returns, on rank 0, a list of `count` entries
    indexed by global search id; None on the other ranks."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        parts = [local]
    else:
        world = dist.get_world_size()
        parts = [None] * world if dist.get_rank() == 0 else None
        dist.gather_object(dict(local), parts, dst=0)
        if dist.get_rank() != 0:
            return None
    out = [None] * count
    for part in parts:
        for s, (f, x) in part.items():
            if out[s] is not None:
                raise ValueError("search %d reported by two ranks" % s)
            out[s] = (float(f), [float(v) for v in x])
    missing = [s for s in range(count) if out[s] is None]
    if missing:
        raise ValueError("searches without a result: %s" % missing[:8])
    return out


def whole_job_rate(units_per_rank_step, steps, world, max_ms):
    """Units all ranks processed per second, timed by the slowest rank."""
    return units_per_rank_step * steps * world / (max_ms / 1e3)

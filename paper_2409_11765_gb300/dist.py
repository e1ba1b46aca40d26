"""Multi-GPU layout of the batched engine: one process per GPU, independent
searches per rank, no collective on the data path.

The paper's K-Distributed strategy (§3.2.3) runs the descents of every
population level at the same time on disjoint groups of processes. On GPUs the
unit of independence is the search: each rank owns whole searches (weak
scaling: every rank runs its own batch with its own Philox seed), and the only
communication is the timing barrier and the maximum of the per-rank times.
"""
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


def max_over_ranks(value, dist=None, device=None):
    """Largest value over all ranks (the timing rule: the slowest rank)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, world, max_ms):
    """Units all ranks processed per second, timed by the slowest rank."""
    return units_per_rank_step * steps * world / (max_ms / 1e3)

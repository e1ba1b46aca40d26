"""The N > 1 host logic on CPU: two gloo ranks on 127.0.0.1."""
import math
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2409_11765_gb300 import dist as D
from paper_2409_11765_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _batch_costs():
    shapes = W.batch256_shapes()
    return [D.search_cost(n, lam) for n, lam, _ in shapes], shapes


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, lr, w = D.env()
    t_ms = 10.0 + 5.0 * rank                    # the slower rank sets the time
    m = D.max_over_ranks(t_ms, dist)
    lo, hi = D.shard(10, world, rank)
    # cost-balanced ownership of the 256-search batch, and the final gather
    costs, wl = _batch_costs()
    mine = D.assign(costs, world)[rank]
    local = {s: (1000.0 + s, [float(s), -float(s)]) for s in mine}
    best = D.gather_best(local, len(costs), dist)
    # the global stop flag: rank 1 alone is below the target
    stop = D.stop_flag(1e-9 if rank == 1 else 5.0, 1e-8, dist)
    nostop = D.stop_flag(1.0 + rank, 1e-8, dist)
    dist.barrier()
    out[rank] = (r, lr, w, m, lo, hi, D.rank_seed(20240918, rank), mine, best, stop, nostop)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, lr, w, m, lo, hi, seed, mine, best, stop, nostop) in res.items():
        assert (r, lr, w) == (rank, rank, world)
        assert m == 15.0                          # max over ranks
        assert stop is True and nostop is False   # the flag is the same on every rank
    spans = sorted((v[4], v[5]) for v in res.values())
    assert spans == [(0, 5), (5, 10)]
    assert res[0][6] != res[1][6]
    # the two ranks own disjoint searches covering the batch
    owned = sorted(res[0][7] + res[1][7])
    assert owned == list(range(256))
    # rank 0 holds every search's result, indexed by global id; rank 1 none
    best = res[0][8]
    assert res[1][8] is None
    assert len(best) == 256
    for s, (f, x) in enumerate(best):
        assert f == 1000.0 + s and x == [float(s), -float(s)]


@pytest.mark.parametrize("count,world", [(10, 1), (10, 3), (256, 8), (3, 4)])
def test_shard_covers_every_search_once(count, world):
    seen = []
    for r in range(world):
        lo, hi = D.shard(count, world, r)
        seen.extend(range(lo, hi))
    assert seen == list(range(count))


def test_lazy_interval_matches_oracle():
    from oracle.params import Params
    for n in (2, 10, 50, 100, 200, 500, 1000, 2000, 4096):
        for lam in (W.default_lambda(n), 2 * W.default_lambda(n), 256, 1024, 8192):
            assert D.lazy_eig_interval(n, lam) == Params(n, lam).g_eig, (n, lam)


@pytest.mark.parametrize("world", [2, 4, 8])
def test_assign_balances_batch256(world):
    costs, wl = _batch_costs()
    owned = D.assign(costs, world)
    assert sorted(s for o in owned for s in o) == list(range(len(costs)))
    loads = [sum(costs[s] for s in o) for o in owned]
    avg = sum(costs) / world
    # greedy longest-first: no rank exceeds the average by more than the
    # largest single search (Graham's bound for list scheduling)
    assert max(loads) <= avg + max(costs)
    # and it beats the contiguous count split on this uneven batch
    split = [sum(costs[D.shard(len(costs), world, r)[0]:D.shard(len(costs), world, r)[1]])
             for r in range(world)]
    assert max(loads) <= max(split)
    assert max(loads) / avg < 1.1


def test_assign_small_cases():
    assert D.assign([5.0, 1.0, 1.0, 1.0, 1.0, 1.0], 2) == [[0], [1, 2, 3, 4, 5]]
    assert D.assign([], 3) == [[], [], []]
    assert D.assign([1.0, 1.0], 4) == [[0], [1], [], []]


def test_gather_single_process():
    best = D.gather_best({1: (2.0, [0.5]), 0: (3.0, [1.5])}, 2)
    assert best == [(3.0, [1.5]), (2.0, [0.5])]
    with pytest.raises(ValueError):
        D.gather_best({0: (1.0, [0.0])}, 2)
    assert D.stop_flag(1e-9, 1e-8) and not D.stop_flag(1.0, 1e-8)
    assert math.isinf(D.global_min(math.inf))


def test_whole_job_rate():
    assert D.whole_job_rate(17391, 100, 2, 1000.0) == 17391 * 100 * 2

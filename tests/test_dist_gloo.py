"""The N > 1 host logic on CPU: two gloo ranks on 127.0.0.1."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2409_11765_gb300 import dist as D


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, lr, w = D.env()
    t_ms = 10.0 + 5.0 * rank                    # the slower rank sets the time
    m = D.max_over_ranks(t_ms, dist)
    lo, hi = D.shard(10, world, rank)
    dist.barrier()
    out[rank] = (r, lr, w, m, lo, hi, D.rank_seed(20240918, rank))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for rank, (r, lr, w, m, lo, hi, seed) in res.items():
        assert (r, lr, w) == (rank, rank, world)
        assert m == 15.0                          # max over ranks
    spans = sorted((v[4], v[5]) for v in res.values())
    assert spans == [(0, 5), (5, 10)]
    assert res[0][6] != res[1][6]


@pytest.mark.parametrize("count,world", [(10, 1), (10, 3), (256, 8), (3, 4)])
def test_shard_covers_every_search_once(count, world):
    seen = []
    for r in range(world):
        lo, hi = D.shard(count, world, r)
        seen.extend(range(lo, hi))
    assert seen == list(range(count))


def test_whole_job_rate():
    assert D.whole_job_rate(17391, 100, 2, 1000.0) == 17391 * 100 * 2

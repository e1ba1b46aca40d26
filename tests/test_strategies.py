"""Host logic of the restart strategies (§3.2.2, §3.2.3) and of the ERT /
ECDF measures (§4.2), pinned on hand-worked cases."""
import math

import pytest

from paper_2409_11765_gb300 import strategies as S


def test_ert_is_total_time_over_successes():
    # three runs: hit at 10, no hit within a budget of 20, hit at 30
    assert S.ert([10, 20, 30], [True, False, True]) == pytest.approx(30.0)
    # all successful: the mean hitting time
    assert S.ert([4, 6], [True, True]) == pytest.approx(5.0)
    assert S.ert([5, 7], [False, False]) == math.inf


def _run(hits, total):
    return {"hits": [None if h is None else {"device_ms": h, "gens": 0, "evals": 0} for h in hits],
            "total": {"device_ms": total, "gens": 0, "evals": 0}}


def test_ert_table_and_ecdf():
    targets = (1.0, 0.1)
    runs = [_run([2.0, None], 10.0), _run([4.0, 8.0], 8.0)]
    tab = S.ert_table(runs, targets)
    # target 1: (2 + 4) / 2; target 0.1: (10 + 8) / 1
    assert tab[0]["ert"] == pytest.approx(3.0) and tab[0]["successes"] == 2
    assert tab[1]["ert"] == pytest.approx(18.0) and tab[1]["successes"] == 1
    # (target, run) pairs hit by t: {2, 4, 8} of four pairs
    assert S.ecdf(runs, targets, [1.0, 2.0, 5.0, 8.0, 100.0]) == [0.0, 0.25, 0.5, 0.75, 0.75]


def test_kreplicated_tree_merges_sibling_pairs():
    t = S.KReplicatedTree(3)
    assert t.on_stopped(1) == []          # sibling 0 still running
    assert t.on_stopped(0) == [0]         # (0, 1) -> descent of 2 lambda in search 0
    assert t.level[0] == 1 and t.retired[1]
    assert t.on_stopped(3) == []
    assert t.on_stopped(2) == [2]         # (2, 3) -> level 1 in search 2
    assert t.on_stopped(0) == []          # level-1 sibling (search 2) still running
    assert t.on_stopped(2) == [0]         # level 2 in search 0
    assert t.level[0] == 2 and t.retired[2]
    for s in (4, 5, 6, 7):
        t.on_stopped(s)
    assert t.level[4] == 1 and t.level[6] == 1
    assert t.on_stopped(4) == []
    assert t.on_stopped(6) == [4]         # level 2 in search 4
    assert t.on_stopped(4) == []          # the level-2 sibling (search 0) runs
    assert t.on_stopped(0) == [0]         # root: level 3 = 2^3 lambda_start
    assert t.level[0] == 3
    assert t.on_stopped(0) == []          # the root's stop ends the schedule
    # how far each search's lambda can grow
    assert [t.max_lambda_multiple(s) for s in range(8)] == [8, 1, 2, 1, 4, 1, 2, 1]


def test_candidates_per_generation_match_between_strategies():
    # K-Replicated with 2^(k+1) leaves uses one lambda_start more per
    # generation than K-Distributed's levels 2^0 .. 2^k (the paper's 512 / 511)
    for k in range(1, 10):
        kdist = sum(1 << j for j in range(k + 1))
        krep = 1 << (k + 1)
        assert krep - kdist == 1

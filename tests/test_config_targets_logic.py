"""The accounting of tests/config_targets.py on a scripted stand-in for the
engine (no GPU): candidates summed over the live searches of every generation
with each one's current lambda, the generation of the first search that
reports a reached target, and a run over the wall budget stopping."""
import numpy as np

import config_targets as CT
from paper_2409_11765_gb300 import workloads as W


class _Script:
    """Per search: (lambda0, generations of each descent, hits the target at
    the end of the last one). A descent's end doubles lambda (sequential
    IPOP) and the search ends after its last descent."""

    def __init__(self, plans):
        self.plans = plans

    def cmaes_default_options(self, **kw):
        return kw

    def cmaes_create_batch(self, ns, lams, x0s, sigma0s, seed, opt):
        return {"s": [dict(lam=p[0], desc=0, gen=0, done=0, flags=0) for p in self.plans],
                "best": [1.0] * len(self.plans)}

    def cmaes_set_problem(self, h, *a):
        pass

    def cmaes_query(self, h, s):
        st = h["s"][s]
        return dict(lam=st["lam"], gen=st["gen"], restart=st["desc"], flags=st["flags"], done=st["done"])

    def cmaes_step_batch(self, h, g):
        for _ in range(g):
            for s, st in enumerate(h["s"]):
                if st["done"]:
                    continue
                lam0, lengths, hits = self.plans[s]
                st["gen"] += 1
                if st["gen"] == lengths[st["desc"]]:
                    if st["desc"] == len(lengths) - 1:
                        st["done"] = 1
                        st["flags"] = 1 if hits else 2
                        h["best"][s] = 1e-9 if hits else 1.0
                    else:
                        st["desc"] += 1
                        st["gen"] = 0
                        st["lam"] *= 2
                        st["flags"] = 4

    def cmaes_sync(self, h):
        pass

    def cmaes_best(self, h, s, n):
        return np.zeros(n), h["best"][s]

    def cmaes_destroy(self, h):
        pass


def test_candidates_and_hit_generation_across_restarts():
    wl = W.ellipsoid_n10()
    eng = _Script([(10, [3, 4, 5], True)])  # descents of 3, 4, 5 generations at lambda 10, 20, 40
    c = CT.counting_run(eng, wl, 0, 1, 1000, 60.0)
    assert c["hit_gen"] == 12 and c["gens"] == 12
    assert c["hit_cand"] == 3 * 10 + 4 * 20 + 5 * 40
    el, best = CT.timed_run(eng, wl, 0, 1, c["gens"], 5)
    assert best == [b for _, b in c["best"]]


def test_batch_counts_only_live_searches():
    wl = W.rastrigin_n100_ipop(concurrent=True, levels=3)
    eng = _Script([(17, [2], False), (34, [5], True), (68, [9], False)])
    c = CT.counting_run(eng, wl, 0, 1, 1000, 60.0)
    # search 1 hits at generation 5; with ten or fewer searches the job ends there
    assert c["hit_gen"] == 5
    assert c["hit_cand"] == 2 * 17 + 5 * 34 + 5 * 68


def test_generation_budget_without_a_hit():
    wl = W.ellipsoid_n10()
    eng = _Script([(10, [1000], True)])
    c = CT.counting_run(eng, wl, 0, 1, 25, 60.0)
    assert c["hit_gen"] is None and c["gens"] == 25 and c["cand"] == 250


def test_markdown_table():
    row = dict(config="c", precision="tf32", f_target=1e-8, reached=True, generations=12,
               candidates=310, seconds=0.5, cand_per_s=620.0, best_f_fp64=9e-9, searches=1,
               searches_at_target=1, descents=[3])
    lines = CT.markdown([row]).splitlines()
    assert len(lines) == 3 and lines[2].startswith("| c | TF32 | 1e-08 | yes | 12 | 310 |")

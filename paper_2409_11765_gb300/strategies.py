"""Parallel restart strategies of the paper on one engine, and the measures the
paper compares them with.

K-Distributed (§3.2.3): the population levels lambda_start * 2^k, k = 0..kmax,
run concurrently as one batch, each level restarting at its own size after a
stop (ipop_double = 0). This is the benchmark's layout.

K-Replicated (§3.2.2): 2^kmax descents of lambda_start run concurrently; when
two sibling descents have both stopped, one descent of twice the population
takes over their resources, up to a single descent of 2^kmax * lambda_start
(a binary tree over the initial descents). On the engine the searches are
created with restart_hold = 1 and ipop_double = 1: a search whose descent
stops pauses (done = 2), and the host restarts the left sibling with lambda
doubled once both siblings are paused (`KReplicatedTree`).

Quality and time (§4.2): for targets eps on f - f_opt (f_opt = 0 for the
built-in objectives) the hitting time of a run is the first time its best
value so far is below eps. ERT (Hansen et al.) = the sum over runs of the time
each spent (the hitting time, or the whole budget if it never hit) divided by
the number of runs that hit; infinite without a success. The ECDF at time t is
the fraction of (target, run) pairs hit by time t.

Command line (one GB300):
    python -m paper_2409_11765_gb300.strategies --objective rastrigin --n 40 \\
        --lam-start 12 --kmax 4 --seeds 10 --max-gens 4000
prints one JSON line with the ERT of both strategies per target, their ratio,
the ECDF on a time grid and each strategy's candidates/s.
"""
import argparse
import json
import math

import numpy as np

TARGETS = (1e2, 10 ** 1.5, 1e1, 10 ** 0.5, 1e0, 1e-2, 1e-4, 1e-6, 1e-8)


def ert(spent, hit):
    """ERT over runs: spent[r] = time run r ran until it hit (or its whole
    budget), hit[r] = whether it hit. Returns inf when no run hit."""
    succ = sum(1 for h in hit if h)
    if succ == 0:
        return math.inf
    return float(sum(spent)) / succ


def ert_table(runs, targets, key="device_ms"):
    """runs: list of run records (see run_strategy); per target the ERT in
    the run records' time unit `key` and the number of successful runs."""
    table = []
    for j, eps in enumerate(targets):
        spent, hit = [], []
        for r in runs:
            h = r["hits"][j]
            hit.append(h is not None)
            spent.append(h[key] if h is not None else r["total"][key])
        table.append({"target": eps, "ert": ert(spent, hit), "successes": sum(hit)})
    return table


def ecdf(runs, targets, grid, key="device_ms"):
    """Fraction of (target, run) pairs hit by each time of `grid`."""
    times = []
    for r in runs:
        for j in range(len(targets)):
            h = r["hits"][j]
            times.append(h[key] if h is not None else math.inf)
    times = np.asarray(times, dtype=np.float64)
    return [float(np.mean(times <= t)) for t in grid]


class KReplicatedTree:
    """Host side of K-Replicated over 2^kmax leaves (search s starts at
    lambda_start). Node (level L, first leaf a) runs in search a. When both
    children of a node have stopped, the node's descent starts in its left
    child's search with twice the population; the right child's search stays
    paused. After the root's descent nothing restarts."""

    def __init__(self, kmax):
        self.kmax = kmax
        self.leaves = 1 << kmax
        self.level = [0] * self.leaves      # level of the descent each search runs
        self.stopped = [False] * self.leaves
        self.retired = [False] * self.leaves

    def on_stopped(self, s):
        """Records that search s's descent stopped; returns the searches to
        restart now (each with lambda doubled)."""
        self.stopped[s] = True
        L = self.level[s]
        if L >= self.kmax:
            return []                         # the root finished
        left = s & ~((1 << (L + 1)) - 1)
        right = left + (1 << L)
        if not (self.stopped[left] and self.level[left] == L
                and self.stopped[right] and self.level[right] == L):
            return []
        # both children of the level L + 1 node have stopped: the node's
        # descent runs in the left child's search, the right one retires
        self.retired[right] = True
        self.level[left] = L + 1
        self.stopped[left] = False
        return [left]

    def max_lambda_multiple(self, s):
        """Largest lambda / lambda_start search s can reach: 2^(trailing zeros)."""
        if s == 0:
            return self.leaves
        return s & -s


def _problem(objective, n, seed):
    from . import workloads as W
    kind = {"ellipsoid": W.ELLIPSOID, "rastrigin": W.RASTRIGIN, "sphere": W.SPHERE}[objective]
    return W.make_problem(kind, n, seed, 7, cond=1e6)


def run_strategy(kind, objective, n, lam_start, kmax, seed, precision=1, max_gens=4000,
                 check_every=10, targets=TARGETS, box=(-5.0, 5.0), sigma0=None):
    """One run of a strategy on a seeded instance; returns the best-so-far
    trace and the hitting times (device ms, generations and evaluations)."""
    import paper_2409_11765_gb300 as eng
    from . import workloads as W
    prob = _problem(objective, n, W.SEED)
    lo, hi = box
    sigma0 = sigma0 if sigma0 is not None else 0.25 * (hi - lo)
    if kind == "kdistributed":
        lams = [lam_start << k for k in range(kmax + 1)]
        opt = eng.cmaes_default_options(precision=precision, f_target=min(targets), box_lo=lo,
                                        box_hi=hi, max_restarts=255, ipop_double=0)
        tree = None
    elif kind == "kreplicated":
        lams = [lam_start] * (1 << kmax)
        opt = eng.cmaes_default_options(precision=precision, f_target=min(targets), box_lo=lo,
                                        box_hi=hi, max_restarts=kmax, ipop_double=1,
                                        restart_hold=1)
        tree = KReplicatedTree(kmax)
    else:
        raise ValueError(kind)
    count = len(lams)
    x0s = [W.start_point(n, lo, hi, seed, 1000 + s) for s in range(count)]
    h = eng.cmaes_create_batch([n] * count, lams, x0s, [sigma0] * count, seed, opt)
    try:
        for s in range(count):
            eng.cmaes_set_problem(h, s, prob.kind, prob.Q, prob.lamdiag, prob.xstar)
        eng.cmaes_set_profiling(h, True)
        eng.cmaes_phase_times(h, reset=True)
        dev_ms = 0.0
        gens = 0
        evals = 0
        trace = []
        seen_paused = [False] * count
        while gens < max_gens:
            q = [eng.cmaes_query(h, s) for s in range(count)]
            running = [s for s in range(count) if q[s]["done"] == 0]
            if not running:
                break
            step = min(check_every, max_gens - gens)
            eng.cmaes_step_batch(h, step)
            ms, _ = eng.cmaes_phase_times(h, reset=True)
            dev_ms += sum(ms.values())
            gens += step
            evals += step * sum(q[s]["lam"] for s in running)
            best = min(eng.cmaes_best(h, s, n)[1] for s in range(count))
            trace.append({"device_ms": dev_ms, "gens": gens, "evals": evals, "best": best})
            if best < min(targets):
                break
            if tree is not None:
                for s in range(count):
                    d = eng.cmaes_query(h, s)["done"]
                    if d == 2 and not seen_paused[s]:
                        seen_paused[s] = True
                        for r in tree.on_stopped(s):
                            eng.cmaes_restart(h, r)
                            seen_paused[r] = False
    finally:
        eng.cmaes_destroy(h)
    hits = []
    for eps in targets:
        hit = next((t for t in trace if t["best"] < eps), None)
        hits.append(None if hit is None else {k: hit[k] for k in ("device_ms", "gens", "evals")})
    total = trace[-1] if trace else {"device_ms": 0.0, "gens": 0, "evals": 0}
    return {"kind": kind, "seed": seed, "hits": hits,
            "total": {k: total[k] for k in ("device_ms", "gens", "evals")},
            "best": total.get("best", math.inf),
            "candidates_per_s": (total["evals"] / (total["device_ms"] * 1e-3)
                                 if total["device_ms"] > 0 else 0.0)}


def compare(objective, n, lam_start, kmax, seeds, precision=1, max_gens=4000, check_every=10):
    """Both strategies over the same seeds. K-Replicated gets 2^(kmax + 1)
    initial descents so that its candidates per generation (2^(kmax+1)
    lambda_start) match K-Distributed's (2^(kmax+1) - 1) lambda_start, as in
    the paper's comparison (§4.1)."""
    out = {"objective": objective, "n": n, "lam_start": lam_start, "kmax_distributed": kmax,
           "kmax_replicated": kmax + 1, "seeds": list(seeds), "targets": list(TARGETS)}
    runs = {"kdistributed": [], "kreplicated": []}
    for seed in seeds:
        runs["kdistributed"].append(run_strategy("kdistributed", objective, n, lam_start, kmax,
                                                 seed, precision, max_gens, check_every))
        runs["kreplicated"].append(run_strategy("kreplicated", objective, n, lam_start, kmax + 1,
                                                seed, precision, max_gens, check_every))
    for kind, rs in runs.items():
        out[kind] = {"ert_ms": ert_table(rs, TARGETS, "device_ms"),
                     "ert_evals": ert_table(rs, TARGETS, "evals"),
                     "candidates_per_s": float(np.mean([r["candidates_per_s"] for r in rs])),
                     "runs": [{"seed": r["seed"], "best": r["best"], **r["total"]} for r in rs]}
    out["speedup_distributed_over_replicated"] = [
        (a["ert"] / b["ert"]) if math.isfinite(a["ert"]) and math.isfinite(b["ert"]) else None
        for a, b in zip(out["kreplicated"]["ert_ms"], out["kdistributed"]["ert_ms"])]
    tmax = max(r["total"]["device_ms"] for rs in runs.values() for r in rs)
    grid = [tmax * f for f in (0.01, 0.03, 0.1, 0.3, 1.0)]
    out["ecdf_grid_ms"] = grid
    for kind, rs in runs.items():
        out[kind]["ecdf"] = ecdf(rs, TARGETS, grid, "device_ms")
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--objective", default="rastrigin", choices=("rastrigin", "ellipsoid", "sphere"))
    ap.add_argument("--n", type=int, default=40)
    ap.add_argument("--lam-start", type=int, default=12)
    ap.add_argument("--kmax", type=int, default=4)
    ap.add_argument("--seeds", type=int, default=10)
    ap.add_argument("--max-gens", type=int, default=4000)
    ap.add_argument("--check-every", type=int, default=10)
    ap.add_argument("--precision", default="tf32", choices=("fp64", "tf32", "bf16"))
    a = ap.parse_args()
    prec = {"fp64": 0, "tf32": 1, "bf16": 2}[a.precision]
    res = compare(a.objective, a.n, a.lam_start, a.kmax, range(1, a.seeds + 1), prec, a.max_gens,
                  a.check_every)
    res["precision"] = a.precision

    def clean(x):
        if isinstance(x, float) and not math.isfinite(x):
            return None
        if isinstance(x, dict):
            return {k: clean(v) for k, v in x.items()}
        if isinstance(x, list):
            return [clean(v) for v in x]
        return x
    print(json.dumps(clean(res)))


if __name__ == "__main__":
    main()

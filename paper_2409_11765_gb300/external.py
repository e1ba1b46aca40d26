"""External (host-evaluated) objectives at throughput: the paper's black-box
setting, where f is a costly function the optimiser only calls (§1, §4.1).

`AsyncAskTell` splits the searches of a handle into groups, each on its own
CUDA stream with pinned host buffers. Per generation and group it waits for
the group's points, evaluates f on the host, then enqueues the group's tell
(rank, update, covariance, eigendecomposition, stop) and its next ask
(sampling and the copy of the points back) without waiting. While the host
evaluates one group, the device updates and samples the others, so with two
groups of similar size the device time hides behind the host evaluation.

Command line (one GB300, the K-Distributed Rastrigin n = 100 batch with f
evaluated on the host cores with numpy):
    python -m paper_2409_11765_gb300.external --gens 20
prints one JSON line with candidates/s for synchronous per-search ask/tell,
the asynchronous path with one group, and with two overlapped groups.
"""
import argparse
import json
import time

import numpy as np


def host_objective(kind, Q, lamdiag, xstar):
    """The built-in objectives written for the host: X is n x m, returns m
    values (the caller's black box in the benchmark)."""
    n = xstar.shape[0]

    def rastrigin(X):
        U = Q @ (X - xstar[:, None])
        return 10.0 * n + np.sum(U * U - 10.0 * np.cos(2.0 * np.pi * U), axis=0)

    def ellipsoid(X):
        U = Q @ (X - xstar[:, None])
        return np.sum(lamdiag[:, None] * U * U, axis=0)

    def sphere(X):
        R = X - xstar[:, None]
        return np.sum(R * R, axis=0)

    return {1: ellipsoid, 2: rastrigin, 3: sphere}[kind]


class AsyncAskTell:
    """Asynchronous ask / tell over groups of searches [a, b) of a handle."""

    def __init__(self, h, ns, lam_caps, groups):
        import torch
        import paper_2409_11765_gb300 as eng
        self.eng, self.h, self.ns, self.groups = eng, h, list(ns), list(groups)
        self.X = [torch.empty((cap, n), dtype=torch.float64, pin_memory=True)
                  for n, cap in zip(ns, lam_caps)]   # (cap, n) row-major = n x cap column-major
        self.f = [torch.empty(cap, dtype=torch.float64, pin_memory=True) for cap in lam_caps]
        self.ld = [torch.zeros(2 * (b - a), dtype=torch.int32, pin_memory=True) for a, b in groups]
        self.streams = [torch.cuda.Stream() for _ in groups]
        self.pending = [False] * len(groups)

    def ask(self, g):
        a, b = self.groups[g]
        self.eng.cmaes_ask_async(self.h, a, b, [self.X[s].data_ptr() for s in range(a, b)],
                                 self.ld[g].data_ptr(), self.streams[g].cuda_stream)
        self.pending[g] = True

    def tell(self, g):
        a, b = self.groups[g]
        self.eng.cmaes_tell_async(self.h, a, b, [self.f[s].data_ptr() for s in range(a, b)],
                                  self.streams[g].cuda_stream)
        self.pending[g] = False

    def evaluate(self, g, fns):
        """Waits for group g's points and writes f for its running searches;
        returns the number of candidates evaluated."""
        a, b = self.groups[g]
        self.streams[g].synchronize()
        ld = self.ld[g].numpy()
        done = 0
        for s in range(a, b):
            lam, finished = int(ld[2 * (s - a)]), int(ld[2 * (s - a) + 1])
            if finished:
                continue
            Xs = self.X[s].numpy()[:lam].T
            self.f[s].numpy()[:lam] = fns[s](Xs)
            done += lam
        return done

    def run(self, fns, generations):
        """`generations` generations of every group; returns candidates
        evaluated. The last asks stay pending, and a later run continues from
        them."""
        for g in range(len(self.groups)):
            if not self.pending[g]:
                self.ask(g)
        total = 0
        for _ in range(generations):
            for g in range(len(self.groups)):
                total += self.evaluate(g, fns)
                self.tell(g)
                self.ask(g)
        for st in self.streams:
            st.synchronize()
        return total


def run_sync(h, ns, fns, generations):
    """Synchronous per-search ask / tell (cmaes_ask / cmaes_tell)."""
    import paper_2409_11765_gb300 as eng
    total = 0
    for _ in range(generations):
        for s, n in enumerate(ns):
            if eng.cmaes_query(h, s)["done"]:
                continue
            X = eng.cmaes_ask(h, s, n)
            eng.cmaes_tell(h, s, fns[s](X))
            total += X.shape[1]
    return total


def _batch(precision):
    import paper_2409_11765_gb300 as eng
    from . import workloads as W
    wl = W.rastrigin_n100_ipop(concurrent=True)
    opt = eng.cmaes_default_options(precision=precision, f_target=wl.f_target, box_lo=wl.box_lo,
                                    box_hi=wl.box_hi, max_restarts=255, ipop_double=0)
    ns = [s.n for s in wl.searches]
    lams = [s.lam for s in wl.searches]
    h = eng.cmaes_create_batch(ns, lams, [s.x0 for s in wl.searches],
                               [s.sigma0 for s in wl.searches], W.SEED, opt)
    fns = []
    for i, s in enumerate(wl.searches):
        p = s.problem
        eng.cmaes_set_problem(h, i, p.kind, p.Q, p.lamdiag, p.xstar)
        fns.append(host_objective(p.kind, p.Q, p.lamdiag, p.xstar))
    return eng, h, ns, lams, fns


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gens", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="tf32", choices=("fp64", "tf32", "bf16"))
    a = ap.parse_args()
    prec = {"fp64": 0, "tf32": 1, "bf16": 2}[a.precision]
    out = {"workload": "rastrigin-n100-kdist-lam17x2^0..9, f evaluated on the host (numpy)",
           "precision": a.precision, "gens": a.gens}
    # synchronous per-search ask / tell
    eng, h, ns, lams, fns = _batch(prec)
    try:
        run_sync(h, ns, fns, a.warmup)
        t0 = time.perf_counter()
        c = run_sync(h, ns, fns, a.gens)
        out["sync_candidates_per_s"] = c / (time.perf_counter() - t0)
    finally:
        eng.cmaes_destroy(h)
    # host objective alone (the floor of any schedule)
    X = np.random.default_rng(0).standard_normal((ns[0], sum(lams)))
    t0 = time.perf_counter()
    for _ in range(3):
        fns[-1](X)
    out["host_f_candidates_per_s"] = 3 * X.shape[1] / (time.perf_counter() - t0)
    # one group (no overlap) and two groups (the largest level against the rest:
    # 8704 against 8687 candidates per generation)
    for label, groups in (("async_1group", [(0, 10)]), ("async_2groups", [(9, 10), (0, 9)])):
        eng, h, ns, lams, fns = _batch(prec)
        try:
            caps = lams
            pipe = AsyncAskTell(h, ns, caps, groups)
            pipe.run(fns, a.warmup)
            t0 = time.perf_counter()
            c = pipe.run(fns, a.gens)
            out[label + "_candidates_per_s"] = c / (time.perf_counter() - t0)
        finally:
            eng.cmaes_destroy(h)
    print(json.dumps(out))


if __name__ == "__main__":
    main()

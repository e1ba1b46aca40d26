"""The paper-derived configurations run to their f-targets (or their
generation budgets), on the FP64 path and the mixed-precision path.

Not a pytest module: a measurement run on a GPU, whose table is quoted in the
results notes. A configuration whose generations take well under a
millisecond is run twice from the same seed; the engine is deterministic
(fixed-order sums, counter-based normals), so both runs take the same
trajectory, which the script checks on the best values' bits.

  * the counting run steps one generation at a time and reads every search's
    lambda, descent number and stop flags after each generation, so it knows
    the generations and candidates spent until the target was reached;
  * the timed run steps in chunks of generations with no host read in
    between, and its wall time (device work included: every chunk ends with
    cmaes_sync) gives the time to target and candidates/s.

Configurations with long generations (n >= 1000) are run once, one
generation per call, and timed as they are: the host reads then cost little
next to a generation. Each has a wall-time budget; a run that ends on it
reports how far it got.

The best point of every search that reports a reached target is re-evaluated
in FP64 by the oracle's objective, so a mixed-precision hit is a true hit.

    python tests/config_targets.py [--only LABEL-SUBSTRING] [--precision fp64|tf32]
                                   [--json out.json]
    python tests/config_targets.py --markdown out.json     (the table of a saved run)
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

PRECISIONS = (("fp64", 0), ("tf32", 1))


def _configs():
    from paper_2409_11765_gb300 import workloads as W
    # (label, workload, generation budget, wall-seconds budget, timed chunk)
    return [
        ("ellipsoid n=10 lam=10, cond 1e6 (plain CMA-ES)", W.ellipsoid_n10(), 2000, 60.0, 50),
        ("Rastrigin n=100, sequential IPOP lam0=17 x2 per restart, 9 restarts",
         W.rastrigin_n100_ipop(concurrent=False), 10 ** 6, 150.0, 50),
        ("Rastrigin n=100, K-Distributed levels lam=17*2^0..9",
         W.rastrigin_n100_ipop(concurrent=True), 10 ** 6, 150.0, 20),
        ("ellipsoid n=1000 lam=1024, cond 1e6", W.ellipsoid_n1000(), 5000, 200.0, 1),
        ("256-search uneven batch n=50..2000", W.batch256(), 10 ** 6, 60.0, 1),
        ("ellipsoid n=4096 lam=8192, cond 1e4", W.ellipsoid_n4096(), 2000, 60.0, 1),
        ("sphere n=4096 lam=8192 (separable control)", W.ellipsoid_n4096(kind=W.SPHERE),
         2000, 60.0, 1),
    ]


def _handle(eng, wl, prec, seed):
    opt = eng.cmaes_default_options(precision=prec, f_target=wl.f_target, box_lo=wl.box_lo,
                                    box_hi=wl.box_hi, max_restarts=min(wl.max_restarts, 255),
                                    ipop_double=1 if wl.ipop_double else 0)
    h = eng.cmaes_create_batch([s.n for s in wl.searches], [s.lam for s in wl.searches],
                               [s.x0 for s in wl.searches], [s.sigma0 for s in wl.searches],
                               seed, opt)
    for i, s in enumerate(wl.searches):
        p = s.problem
        eng.cmaes_set_problem(h, i, p.kind, p.Q, p.lamdiag, p.xstar)
    return h


def counting_run(eng, wl, prec, seed, max_gens, max_seconds):
    """One generation per call: generations, candidates and descents until the
    first search reaches the target (or the budget ends)."""
    h = _handle(eng, wl, prec, seed)
    S = len(wl.searches)
    try:
        q = [eng.cmaes_query(h, s) for s in range(S)]
        gens, cand, hit_gen, hit_cand = 0, 0, None, None
        t0 = time.perf_counter()
        while gens < max_gens and time.perf_counter() - t0 < max_seconds:
            live = [s for s in range(S) if q[s]["done"] == 0]
            if not live:
                break
            cand += sum(q[s]["lam"] for s in live)
            eng.cmaes_step_batch(h, 1)
            gens += 1
            q = [eng.cmaes_query(h, s) for s in range(S)]
            if hit_gen is None and any(x["flags"] & 1 and x["done"] == 1 for x in q):
                hit_gen, hit_cand = gens, cand
                if S <= 10:          # a single search or the K-Distributed levels: the job is done
                    break
        eng.cmaes_sync(h)
        el = time.perf_counter() - t0
        best = [eng.cmaes_best(h, s, wl.searches[s].n) for s in range(S)]
        return dict(gens=gens, cand=cand, hit_gen=hit_gen, hit_cand=hit_cand, q=q, best=best,
                    seconds=el)
    finally:
        eng.cmaes_destroy(h)


def timed_run(eng, wl, prec, seed, gens, chunk):
    """The same trajectory, `gens` generations in chunks with no host read
    between the generations of a chunk; wall seconds."""
    h = _handle(eng, wl, prec, seed)
    try:
        eng.cmaes_sync(h)
        t0 = time.perf_counter()
        done = 0
        while done < gens:
            g = min(chunk, gens - done)
            eng.cmaes_step_batch(h, g)
            done += g
        eng.cmaes_sync(h)
        el = time.perf_counter() - t0
        best = [eng.cmaes_best(h, s, wl.searches[s].n)[1] for s in range(len(wl.searches))]
        return el, best
    finally:
        eng.cmaes_destroy(h)


def fp64_recheck(wl, best):
    from oracle import objectives
    out = []
    for s, (x, f) in enumerate(best):
        p = wl.searches[s].problem
        out.append(float(objectives.evaluate(p.kind, x[:, None], p.Q, p.lamdiag, p.xstar)[0]))
    return out


def markdown(rows):
    """The results table as it appears in the results notes."""
    out = ["| configuration | path | target | reached | generations | candidates | time (s) | "
           "candidates/s | best f (FP64 re-evaluated) | descents |",
           "|---|---|---:|---|---:|---:|---:|---:|---:|---|"]
    for r in rows:
        reached = "yes" if r["reached"] else "no (budget)"
        if r["searches"] > 10:
            reached = "%d of %d searches" % (r["searches_at_target"], r["searches"])
        d = r["descents"]
        ds = str(d[0]) if len(d) == 1 else ("levels " + ",".join(map(str, d)))
        out.append("| %s | %s | %.0e | %s | %d | %d | %.2f | %.3g | %.3e | %s |" % (
            r["config"], r["precision"].upper(), r["f_target"], reached, r["generations"],
            r["candidates"], r["seconds"], r["cand_per_s"], r["best_f_fp64"], ds))
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", default="")
    ap.add_argument("--precision", choices=["fp64", "tf32"], default=None)
    ap.add_argument("--json", default="")
    ap.add_argument("--seed", type=int, default=20240918)
    ap.add_argument("--markdown", default="", help="print the table of a saved --json file and exit")
    args = ap.parse_args()
    if args.markdown:
        with open(args.markdown) as fh:
            print(markdown(json.load(fh)))
        return
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_11765_gb300 as eng
    rows = []
    for label, wl, max_gens, max_s, chunk in _configs():
        if args.only and args.only not in label:
            continue
        for pname, prec in PRECISIONS:
            if args.precision and pname != args.precision:
                continue
            c = counting_run(eng, wl, prec, args.seed, max_gens, max_s)
            gens = c["hit_gen"] if c["hit_gen"] is not None else c["gens"]
            cand = c["hit_cand"] if c["hit_cand"] is not None else c["cand"]
            same = None
            if chunk > 1:
                el, tbest = timed_run(eng, wl, prec, args.seed, gens, chunk)
                same = all(a == b for a, (_, b) in zip(tbest, c["best"]))
            else:   # generations long enough that the per-generation reads cost little
                el = c["seconds"]
            fre = fp64_recheck(wl, c["best"])
            hits = [s for s, x in enumerate(c["q"]) if x["flags"] & 1 and x["done"] == 1]
            row = dict(config=label, precision=pname, f_target=wl.f_target,
                       reached=c["hit_gen"] is not None, generations=gens, candidates=cand,
                       seconds=round(el, 3), timed_chunk=chunk, same_trajectory=same,
                       cand_per_s=round(cand / el, 1) if el > 0 else None,
                       best_f=float(min(b[1] for b in c["best"])), best_f_fp64=float(min(fre)),
                       searches=len(wl.searches), searches_at_target=len(hits),
                       hits_true_fp64=all(fre[s] < wl.f_target for s in hits),
                       descents=[x["restart"] + 1 for x in c["q"]][:10],
                       lambdas=[x["lam"] for x in c["q"]][:10])
            rows.append(row)
            print(json.dumps(row), flush=True)
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(rows, fh, indent=1)


if __name__ == "__main__":
    main()

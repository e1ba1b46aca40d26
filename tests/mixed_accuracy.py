"""Measured error of the mixed-precision path against the FP64 oracle, per
state quantity, and the fraction of generations whose selected set (the mu
best candidates, the ones Eq. (2) weights) is identical.

Not a pytest module: a measurement run on a GPU, whose table is quoted in the
design notes. For each configuration shape, G generations are run
teacher-forced: before every generation the handle is loaded with the oracle's
current state, both sides take one generation from it (the same Philox
normals on both sides; the device evaluates f with its mixed-precision
objective, the oracle in FP64), and every state quantity is compared. The
oracle's state then advances (so the trajectory is the oracle's own).

    python tests/mixed_accuracy.py [--gens 20] [--json out.json]
"""
import argparse
import json
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

CASES = [  # (label, n, lambda, objective kind, cond, stream)
    ("ellipsoid n=10 lam=10 (cond 1e6)", 10, 10, 1, 1e6, 0),
    ("Rastrigin n=100 lam=17", 100, 17, 2, 1.0, 1),
    ("Rastrigin n=100 lam=1088", 100, 1088, 2, 1.0, 2),
    ("Rastrigin n=100 lam=8704", 100, 8704, 2, 1.0, 3),
    ("ellipsoid n=1000 lam=1024 (cond 1e6)", 1000, 1024, 1, 1e6, 4),
]


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    d = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (d if d > 0 else 1.0))


def run_case(label, n, lam, kind, cond, stream, prec, gens):
    import paper_2409_11765_gb300 as eng
    from oracle import cmaes, objectives
    from paper_2409_11765_gb300 import workloads as W
    from parity_util import SEED, oracle_problem, oracle_state, state_dict
    p = W.make_problem(kind, n, SEED, 1500 + stream, cond=cond)
    d = W.random_state(n, SEED, 1500 + stream, cond=1e2)
    st = oracle_state(d, n, lam, 1.0, gen=1)
    opts = cmaes.Options(eig_every=1, max_restarts=0)
    opt = eng.cmaes_default_options(precision=prec, eig_every=1, max_restarts=0)
    h = eng.cmaes_create(n, lam, d["m"], 1.0, SEED, opt)
    err = {k: [] for k in ("x", "f", "m", "p_sigma", "p_c", "sigma", "C", "eigenvalues")}
    same_sel = same_order = 0
    try:
        eng.cmaes_set_problem(h, 0, p.kind, p.Q, p.lamdiag, p.xstar)
        for g in range(gens):
            eng.cmaes_set_state(h, 0, dict(n=n, lam=lam, sigma=st.sigma, m=st.m, ps=st.ps, pc=st.pc,
                                           C=st.C, B=st.B, D=st.D, gen=st.gen))
            eng.cmaes_step_batch(h, 1)
            X, f, order = eng.cmaes_get_generation(h, 0, n)
            s = eng.cmaes_get_state(h, 0, n)
            rec = cmaes.generation(st, SEED, 0, oracle_problem(p), opts)
            mag = objectives.magnitude(p.kind, rec["X"], p.Q, p.lamdiag, p.xstar)
            mu = lam // 2
            err["x"].append(rel(X, rec["X"]))
            err["f"].append(float(np.max(np.abs(f - rec["f"]) / mag)))
            err["m"].append(rel(s["m"], st.m))
            err["p_sigma"].append(rel(s["ps"], st.ps))
            err["p_c"].append(rel(s["pc"], st.pc))
            err["sigma"].append(abs(s["sigma"] / st.sigma - 1.0))
            err["C"].append(float(np.linalg.norm(s["C"] - st.C, 2) / np.linalg.norm(st.C, 2)))
            err["eigenvalues"].append(float(np.max(np.abs(np.sort(s["D"] ** 2) - np.sort(st.D ** 2)))
                                            / np.max(st.D ** 2)))
            same_sel += set(order[:mu].tolist()) == set(rec["order"][:mu].tolist())
            same_order += bool(np.array_equal(order, rec["order"]))
            if st.done:
                break
    finally:
        eng.cmaes_destroy(h)
    done = len(err["x"])
    return {"case": label, "precision": {1: "tf32", 2: "bf16"}[prec], "generations": done,
            "max_rel_error": {k: max(v) for k, v in err.items()},
            "median_rel_error": {k: float(np.median(v)) for k, v in err.items()},
            "identical_selected_set": same_sel / done, "identical_rank_order": same_order / done}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gens", type=int, default=20)
    ap.add_argument("--json", default=None)
    a = ap.parse_args()
    import __graft_entry__
    __graft_entry__.build()
    rows = []
    for case in CASES:
        for prec in (1, 2):
            r = run_case(*case, prec, a.gens if case[1] < 1000 else max(4, a.gens // 4))
            rows.append(r)
            print(json.dumps(r), flush=True)
    if a.json:
        with open(a.json, "w") as fh:
            json.dump(rows, fh, indent=1)


if __name__ == "__main__":
    main()

"""Shared helpers of the GPU parity tests: run one teacher-forced generation
through the C ABI and through the oracle from the same state and inputs."""
import math

import numpy as np

import paper_2409_11765_gb300 as eng
from oracle import cmaes, objectives
from paper_2409_11765_gb300 import workloads as W

SEED = 20240918
# FP64 path: normwise relative error bound of every state quantity.
TOL_FP64 = 1e-12


def have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def oracle_problem(p):
    return cmaes.Problem(p.kind, p.xstar, p.Q, p.lamdiag)


def state_dict(d, n, lam, gen=0, restart=0):
    return dict(n=n, lam=lam, sigma=d["sigma"], m=d["m"], ps=d["ps"], pc=d["pc"], C=d["C"],
                B=d["B"], D=d["D"], gen=gen, restart=restart)


def oracle_state(d, n, lam, sigma0, gen=0, restart=0):
    return cmaes.State(n, lam, d["sigma"], d["m"].copy(), sigma0, d["ps"].copy(), d["pc"].copy(),
                       d["C"].copy(), d["B"].copy(), d["D"].copy(), gen=gen, restart=restart)


def teacher_forced(ns, lams, kinds, states, search=0, eig_every=1, gen=3, restart=0,
                   sigma0=1.0, opt_over=None):
    """Batch of searches; search `search` gets states[search] and is compared.

    Returns (gpu, oracle) dicts with X, f, order and the state after one
    generation."""
    count = len(ns)
    probs = [W.make_problem(k, n, SEED, 50 + i) for i, (k, n) in enumerate(zip(kinds, ns))]
    over = dict(eig_every=eig_every, max_restarts=1)
    if opt_over:
        over.update(opt_over)
    opt = eng.cmaes_default_options(**over)
    h = eng.cmaes_create_batch(ns, lams, [st["m"] for st in states], [sigma0] * count, SEED, opt)
    try:
        for i, p in enumerate(probs):
            eng.cmaes_set_problem(h, i, p.kind, p.Q, p.lamdiag, p.xstar)
            eng.cmaes_set_state(h, i, state_dict(states[i], ns[i], lams[i], gen, restart))
        eng.cmaes_step_batch(h, 1)
        eng.cmaes_sync(h)
        X, f, order = eng.cmaes_get_generation(h, search, ns[search])
        g = eng.cmaes_get_state(h, search, ns[search])
        q = eng.cmaes_query(h, search)
    finally:
        eng.cmaes_destroy(h)
    n, lam = ns[search], lams[search]
    st = oracle_state(states[search], n, lam, sigma0, gen, restart)
    opts = cmaes.Options(eig_every=eig_every, max_restarts=1)
    if opt_over:
        for k, v in opt_over.items():
            setattr(opts, k, v)
    rec = cmaes.generation(st, SEED, search, oracle_problem(probs[search]), opts)
    gpu = dict(X=X, f=f, order=order, state=g, query=q)
    ora = dict(X=rec["X"], Y=rec["Y"], f=rec["f"], order=rec["order"], rec=rec, state=st,
               problem=probs[search])
    return gpu, ora


def near_tie_groups(f_sorted, rtol=1e-10):
    """Group ids of the positions of an ascending f list: neighbours whose
    values differ by at most rtol of the larger magnitude (or are both
    non-finite) share a group, so only there may the last bits decide."""
    fs = np.asarray(f_sorted, dtype=np.float64)
    gid = np.zeros(len(fs), dtype=np.int64)
    for i in range(1, len(fs)):
        a, b = fs[i - 1], fs[i]
        if np.isfinite(a) and np.isfinite(b):
            same = abs(b - a) <= rtol * max(abs(a), abs(b))
        else:
            same = not np.isfinite(a) and not np.isfinite(b)
        gid[i] = gid[i - 1] + (0 if same else 1)
    return gid


def check_order(order_gpu, order_ora, f_ora, rtol=1e-10):
    """Rank order bit-exact, except that candidates whose oracle f values are
    within rtol of each other (a near-tie group) may swap among themselves:
    each group's positions must hold the same set of candidates on both sides."""
    og = np.asarray(order_gpu)
    oo = np.asarray(order_ora)
    assert sorted(og.tolist()) == list(range(len(oo))), "rank order is not a permutation"
    gid = near_tie_groups(np.asarray(f_ora)[oo], rtol)
    for g in np.unique(gid):
        pos = np.nonzero(gid == g)[0]
        if len(pos) == 1:
            assert og[pos[0]] == oo[pos[0]], ("rank order differs at", int(pos[0]))
        else:
            assert set(og[pos].tolist()) == set(oo[pos].tolist()), (
                "near-tie group differs at", pos.tolist())


def check_generation(gpu, ora, tol=TOL_FP64, eig=True):
    """Asserts the teacher-forced generation agrees with the oracle."""
    g, st, rec = gpu["state"], ora["state"], ora["rec"]
    n = st.n
    p = ora["problem"]
    assert rel(gpu["X"], ora["X"]) <= tol, ("X", rel(gpu["X"], ora["X"]))
    mag = objectives.magnitude(p.kind, ora["X"], p.Q, p.lamdiag, p.xstar)
    ferr = np.abs(gpu["f"] - ora["f"]) / np.maximum(mag, 1e-300)
    assert ferr.max() <= tol, ("f", ferr.max())
    check_order(gpu["order"], ora["order"], ora["f"])
    # and the device order is the stable ascending order of the device's own f
    fg = np.where(np.isnan(gpu["f"]), np.inf, gpu["f"])[np.asarray(gpu["order"])]
    og = np.asarray(gpu["order"])
    ok = (fg[1:] > fg[:-1]) | ((fg[1:] == fg[:-1]) & (og[1:] > og[:-1]))
    assert ok.all(), "device order is not sorted by (f, index)"
    if st.restart != g["restart"] or st.done != bool(g["done"]):
        raise AssertionError("restart/done differ: gpu %s oracle %s" % (
            (g["restart"], g["done"]), (st.restart, st.done)))
    assert g["gen"] == st.gen and g["lam"] == st.lam and g["flags"] == st.flags, (
        g["gen"], st.gen, g["flags"], st.flags)
    for k in ("m", "ps", "pc"):
        assert rel(g[k], getattr(st, k)) <= tol, (k, rel(g[k], getattr(st, k)))
    assert math.isclose(g["sigma"], st.sigma, rel_tol=tol), ("sigma", g["sigma"], st.sigma)
    assert rel(g["C"], st.C) <= tol, ("C", rel(g["C"], st.C))
    assert np.array_equal(g["C"], g["C"].T), "C not exactly symmetric"
    if st.best_f < math.inf:
        assert math.isclose(g["best_f"], st.best_f, rel_tol=tol, abs_tol=tol * mag.max())
        assert rel(g["best_x"], st.best_x) <= tol
    B, D = g["B"], g["D"]
    if eig:
        ev_g, ev_o = D ** 2, st.D ** 2
        assert np.all(np.diff(ev_g) >= 0), "eigenvalues not ascending"
        assert np.abs(ev_g - ev_o).max() <= tol * ev_o.max(), ("D", np.abs(ev_g - ev_o).max())
        assert np.abs(B.T @ B - np.eye(n)).max() <= 1e-13 * max(n, 10)
        recon = (B * D ** 2) @ B.T
        assert rel(recon, g["C"]) <= tol, ("BD^2B^T", rel(recon, g["C"]))
        # eigenvectors: same canonical representative, to within the
        # conditioning of each one (relative gap to its neighbours)
        for j in range(n):
            others = np.delete(ev_o, j)
            gap = np.min(np.abs(others - ev_o[j])) / ev_o.max() if n > 1 else 1.0
            if gap > 1e-6:
                err = np.abs(B[:, j] - st.B[:, j]).max()
                assert err <= 1e-13 / gap + 1e-13, ("B column", j, err, gap)
    else:
        assert rel(B, st.B) == 0.0 and rel(D, st.D) == 0.0

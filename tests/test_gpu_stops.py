"""Stop tests fired on the device, and the restart each one triggers, against
the oracle (§2.2's stop categories, Algorithm 2's restart).

Each case loads a state from which one stop test fires at the end of the next
generation, runs that generation through the C ABI and through the oracle, and
compares the flags, the done / restart decision and the whole state after it:
for a restart that is lambda doubled or kept, the fresh Philox mean, sigma0,
C = B = I, D = 1, zero paths, generation 0, an empty history and the best point
kept. Also here: a non-finite state is reported as CMAES_ENUMERIC, and a
device wait that gave up (injected from the host) as a sticky CMAES_ETIMEOUT.
"""
import math

import numpy as np
import pytest

from parity_util import SEED, TOL_FP64, check_order, have_gpu, oracle_problem, rel

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]

STOP_FTARGET, STOP_MAXITER, STOP_TOLHISTFUN, STOP_TOLX = 1, 2, 4, 8
STOP_CONDITIONCOV, STOP_NOEFFECTAXIS, STOP_NOEFFECTCOORD, STOP_NONFINITE = 16, 32, 64, 128


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _state(n, seed_stream, cond=1e2):
    from paper_2409_11765_gb300 import workloads as W
    return W.random_state(n, SEED, seed_stream, cond=cond)


def _run(n, lam, kind, d, gen, opts, hist=None, best_f=math.inf, best_x=None, sigma0=1.0,
         restart=0):
    """One generation from state d on both sides. Returns (gpu, oracle, status)
    where status is the error status the engine reported at the sync after the
    generation (0 if none)."""
    import paper_2409_11765_gb300 as eng
    from oracle import cmaes
    from paper_2409_11765_gb300 import workloads as W
    p = W.make_problem(kind, n, SEED, 800 + n)
    h = eng.cmaes_create(n, lam, np.zeros(n), sigma0, SEED, eng.cmaes_default_options(**opts))
    status = 0
    try:
        eng.cmaes_set_problem(h, 0, p.kind, p.Q, p.lamdiag, p.xstar)
        sd = dict(n=n, lam=lam, sigma=d["sigma"], m=d["m"], ps=d["ps"], pc=d["pc"], C=d["C"],
                  B=d["B"], D=d["D"], gen=gen, restart=restart, best_f=best_f)
        if best_x is not None:
            sd["best_x"] = best_x
        if hist is not None:
            sd["hist"] = np.asarray(hist, dtype=np.float64)
        eng.cmaes_set_state(h, 0, sd)
        eng.cmaes_step_batch(h, 1)
        try:
            eng.cmaes_sync(h)
        except eng.CmaesError as e:
            status = e.status
        g = eng.cmaes_get_state(h, 0, n)
        q = eng.cmaes_query(h, 0)
        gen_panel = None
        if q["lam"] == lam:
            gen_panel = eng.cmaes_get_generation(h, 0, n)
    finally:
        eng.cmaes_destroy(h)
    st = cmaes.State(n, lam, d["sigma"], d["m"].copy(), sigma0, d["ps"].copy(), d["pc"].copy(),
                     d["C"].copy(), d["B"].copy(), d["D"].copy(), gen=gen, restart=restart)
    st.best_f = best_f
    if best_x is not None:
        st.best_x = np.array(best_x, dtype=np.float64)
    if hist is not None:
        st.hist = list(hist)
    o = cmaes.Options()
    for k, v in opts.items():
        setattr(o, k, v)
    rec = cmaes.generation(st, SEED, 0, oracle_problem(p), o)
    return g, q, gen_panel, st, rec, status


def _compare_after(g, q, gen_panel, st, rec, n):
    """The device's decision and state after the generation against the
    oracle's."""
    assert g["flags"] == st.flags, ("flags", g["flags"], st.flags)
    assert bool(g["done"]) == st.done, ("done", g["done"], st.done)
    assert g["restart"] == st.restart and g["lam"] == st.lam and g["gen"] == st.gen
    assert q["flags"] == st.flags and q["lam"] == st.lam
    if gen_panel is not None:
        X, f, order = gen_panel
        fin = np.isfinite(rec["f"])
        if fin.all():
            assert rel(X, rec["X"]) <= TOL_FP64
            check_order(order, rec["order"], rec["f"])
    if st.restart and not st.done and st.gen == 0:
        # a fresh descent: exact reset values, the restart mean from Philox
        assert np.abs(g["m"] - st.m).max() <= 1e-15 * max(1.0, np.abs(st.m).max())
        assert g["sigma"] == st.sigma
        assert np.array_equal(g["C"], np.eye(n)) and np.array_equal(g["B"], np.eye(n))
        assert np.array_equal(g["D"], np.ones(n))
        assert not g["ps"].any() and not g["pc"].any()
        assert len(g["hist"]) == 0 == len(st.hist)
    else:
        for k in ("m", "ps", "pc", "C"):
            assert rel(g[k], getattr(st, k)) <= TOL_FP64, k
        assert math.isclose(g["sigma"], st.sigma, rel_tol=TOL_FP64)
    if math.isfinite(st.best_f):
        assert math.isclose(g["best_f"], st.best_f, rel_tol=TOL_FP64)
        assert rel(g["best_x"], st.best_x) <= TOL_FP64
    else:
        assert not math.isfinite(g["best_f"])


@pytest.mark.parametrize("double", [1, 0])
def test_maxiter_fires_and_restarts(double):
    from oracle.params import Params
    n, lam = 6, 10
    d = _state(n, 900)
    gen = Params(n, lam).max_iter - 1     # the generation counter reaches MaxIter
    r = _run(n, lam, 1, d, gen, dict(max_restarts=3, ipop_double=double, eig_every=1))
    g, q, panel, st, rec, status = r
    assert st.flags & STOP_MAXITER and st.restart == 1 and status == 0
    assert st.lam == (2 * lam if double else lam)
    _compare_after(*r[:5], n)


def test_ftarget_ends_the_search():
    n, lam = 6, 10
    d = _state(n, 901)
    r = _run(n, lam, 1, d, 3, dict(max_restarts=3, f_target=1e30, eig_every=1))
    g, q, panel, st, rec, status = r
    assert st.flags & STOP_FTARGET and st.done and st.restart == 0
    _compare_after(*r[:5], n)


def test_tolhistfun_fires_when_history_is_full():
    from oracle.params import Params
    n, lam = 6, 10
    p = Params(n, lam)
    d = _state(n, 902)
    hist = list(np.linspace(5.0, 6.0, p.hist_len - 1))   # one short of full
    r = _run(n, lam, 1, d, 3, dict(max_restarts=2, tol_hist_fun=1e300, eig_every=1), hist=hist)
    g, q, panel, st, rec, status = r
    assert st.flags == STOP_TOLHISTFUN and st.restart == 1
    _compare_after(*r[:5], n)
    # one more entry short: the history is not full yet, nothing fires
    r = _run(n, lam, 1, d, 3, dict(max_restarts=2, tol_hist_fun=1e300, eig_every=1),
             hist=hist[1:])
    assert r[3].flags == 0 and r[0]["flags"] == 0
    _compare_after(*r[:5], n)


def test_tolx_fires_on_a_tiny_step_size():
    n, lam = 6, 10
    d = _state(n, 903)
    d["sigma"] = 1e-15
    r = _run(n, lam, 1, d, 3, dict(max_restarts=2, eig_every=1))
    g, q, panel, st, rec, status = r
    assert st.flags & STOP_TOLX and st.restart == 1
    _compare_after(*r[:5], n)


def test_conditioncov_fires_without_eig():
    from paper_2409_11765_gb300 import workloads as W
    n, lam = 6, 10
    d = _state(n, 904)
    D2 = np.array([1.0, 3.0, 10.0, 1e3, 1e8, 1e15])
    B = W.haar_orthogonal(n, W.rng_for(SEED, 904))
    C = (B * D2[None, :]) @ B.T
    d.update(B=B, D=np.sqrt(D2), C=0.5 * (C + C.T))
    r = _run(n, lam, 1, d, 3, dict(max_restarts=2, eig_every=1000))
    g, q, panel, st, rec, status = r
    assert st.flags & STOP_CONDITIONCOV and st.restart == 1
    _compare_after(*r[:5], n)


@pytest.mark.parametrize("gen", [3, 4])
def test_noeffect_axis_and_coord(gen):
    n, lam = 4, 8
    d = _state(n, 905)
    d["m"] = np.array([1e20, 0.5, -0.5, 0.25])
    r = _run(n, lam, 3, d, gen, dict(max_restarts=2, eig_every=1))
    g, q, panel, st, rec, status = r
    assert st.flags & STOP_NOEFFECTCOORD and st.restart == 1
    _compare_after(*r[:5], n)


def test_best_point_is_kept_across_the_restart():
    from oracle.params import Params
    n, lam = 6, 10
    d = _state(n, 906)
    gen = Params(n, lam).max_iter - 1
    bx = np.linspace(-1, 1, n)
    r = _run(n, lam, 1, d, gen, dict(max_restarts=3, eig_every=1), best_f=-5.0, best_x=bx)
    g, q, panel, st, rec, status = r
    assert st.restart == 1 and st.best_f == -5.0
    assert g["best_f"] == -5.0 and np.array_equal(g["best_x"], bx)
    _compare_after(*r[:5], n)


def test_restart_budget_spent_ends_the_search():
    from oracle.params import Params
    n, lam = 6, 10
    d = _state(n, 907)
    gen = Params(n, lam).max_iter - 1
    r = _run(n, lam, 1, d, gen, dict(max_restarts=2, eig_every=1), restart=2)
    g, q, panel, st, rec, status = r
    assert st.done and st.restart == 2 and st.flags & STOP_MAXITER
    _compare_after(*r[:5], n)


@pytest.mark.parametrize("what", ["sigma", "m"])
def test_nonfinite_state_is_reported_and_restarted(what):
    import paper_2409_11765_gb300 as eng
    n, lam = 6, 10
    d = _state(n, 908)
    if what == "sigma":
        d["sigma"] = math.nan
    else:
        d["m"] = d["m"].copy()
        d["m"][2] = math.inf
    r = _run(n, lam, 1, d, 3, dict(max_restarts=2, eig_every=1))
    g, q, panel, st, rec, status = r
    assert st.flags & STOP_NONFINITE and st.restart == 1
    assert status == 6                      # CMAES_ENUMERIC, reported at the sync
    assert eng.cmaes_strerror(status) == "non-finite state"
    _compare_after(*r[:5], n)


def test_enumeric_is_reported_once_and_the_handle_stays_usable():
    import paper_2409_11765_gb300 as eng
    n, lam = 6, 10
    d = _state(n, 909)
    h = eng.cmaes_create(n, lam, d["m"], 1.0, SEED, eng.cmaes_default_options(max_restarts=3))
    try:
        eng.cmaes_set_problem(h, 0, eng.OBJ_SPHERE, None, None, np.zeros(n))
        eng.cmaes_set_state(h, 0, dict(n=n, lam=lam, sigma=math.nan, m=d["m"], ps=d["ps"],
                                       pc=d["pc"], C=d["C"], B=d["B"], D=d["D"], gen=1))
        eng.cmaes_step_batch(h, 1)
        with pytest.raises(eng.CmaesError) as e:
            eng.cmaes_sync(h)
        assert e.value.status == 6
        eng.cmaes_sync(h)                   # reported once: the search has restarted
        eng.cmaes_step_batch(h, 3)
        eng.cmaes_sync(h)
        g = eng.cmaes_get_state(h, 0, n)
        assert math.isfinite(g["sigma"]) and np.all(np.isfinite(g["m"])) and g["gen"] == 3
    finally:
        eng.cmaes_destroy(h)


def test_injected_device_timeout_is_sticky():
    import paper_2409_11765_gb300 as eng
    n, lam = 6, 10
    h = eng.cmaes_create(n, lam, np.zeros(n), 1.0, SEED, eng.cmaes_default_options())
    try:
        eng.cmaes_set_problem(h, 0, eng.OBJ_SPHERE, None, None, np.ones(n))
        eng.cmaes_step_batch(h, 1)
        eng.cmaes_sync(h)
        # what a tensor-core or barrier wait does when it gives up: the bit in
        # the device status word, set here from the host
        eng.cmaes_inject_status(h, 1)
        for call in (lambda: eng.cmaes_sync(h), lambda: eng.cmaes_step_batch(h, 1),
                     lambda: eng.cmaes_get_state(h, 0, n), lambda: eng.cmaes_query(h, 0)):
            with pytest.raises(eng.CmaesError) as e:
                call()
            assert e.value.status == 5
        assert "timed out" in eng.cmaes_last_error(h)
    finally:
        eng.cmaes_destroy(h)


def test_mixed_descent_stalled_at_its_resolution_restarts():
    """A mixed (TF32) descent that settles in a local minimum of the rotated
    Rastrigin (n = 100, lambda = 17, the sequential IPOP start) ranks its
    candidates by values whose error (~1e-6 of f, the FP32 epilogue) exceeds
    their differences, so its FP64 best values keep moving by more than the
    absolute TolHistFun tolerance; TolHistFun then compares the window's range
    with 10 x the window's largest |f_mixed - f_FP64| of those best points, and
    the descent restarts within 20,000 generations, as on the FP64 path (before
    that rule it ran on towards MaxIter, ~128,000 generations)."""
    import paper_2409_11765_gb300 as eng
    from paper_2409_11765_gb300 import workloads as W
    wl = W.rastrigin_n100_ipop(concurrent=False)
    s = wl.searches[0]
    res = {}
    for prec in (0, 1):
        opt = eng.cmaes_default_options(precision=prec, f_target=wl.f_target, box_lo=wl.box_lo,
                                        box_hi=wl.box_hi, max_restarts=1, ipop_double=1)
        h = eng.cmaes_create(s.n, s.lam, s.x0, s.sigma0, SEED, opt)
        try:
            p = s.problem
            eng.cmaes_set_problem(h, 0, p.kind, p.Q, p.lamdiag, p.xstar)
            gens = 0
            while gens < 20000:
                eng.cmaes_step_batch(h, 250)
                gens += 250
                q = eng.cmaes_query(h, 0)
                if q["restart"] >= 1 or q["done"]:
                    break
            res[prec] = (gens, q)
        finally:
            eng.cmaes_destroy(h)
    for prec, (gens, q) in res.items():
        assert q["restart"] >= 1 or q["done"], (prec, gens, q)
        assert q["lam"] == 34 or q["done"], (prec, q)

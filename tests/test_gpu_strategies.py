"""Host-driven restarts (restart_hold) and both restart strategies on the
engine, on a small ellipsoid that every strategy solves."""
import math

import numpy as np
import pytest

from parity_util import SEED, have_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def test_restart_hold_pauses_until_the_host_restarts():
    import paper_2409_11765_gb300 as eng
    from paper_2409_11765_gb300 import workloads as W
    n, lam = 8, 6
    p = W.make_problem(W.SPHERE, n, SEED, 3)
    # max_iter = 5 makes every descent stop after 5 generations
    opt = eng.cmaes_default_options(max_restarts=2, ipop_double=1, restart_hold=1, max_iter=5)
    h = eng.cmaes_create(n, lam, np.ones(n), 1.0, SEED, opt)
    try:
        eng.cmaes_set_problem(h, 0, p.kind, p.Q, p.lamdiag, p.xstar)
        eng.cmaes_step_batch(h, 8)
        q = eng.cmaes_query(h, 0)
        assert q["done"] == 2 and q["lam"] == lam and q["restart"] == 0 and q["flags"] & 2
        eng.cmaes_restart(h, 0)
        q = eng.cmaes_query(h, 0)
        assert q["done"] == 0 and q["lam"] == 2 * lam and q["restart"] == 1 and q["gen"] == 0
        eng.cmaes_step_batch(h, 8)
        assert eng.cmaes_query(h, 0)["done"] == 2
        eng.cmaes_restart(h, 0)
        eng.cmaes_step_batch(h, 8)
        q = eng.cmaes_query(h, 0)
        # the restart budget (2) is spent: the search ends for good
        assert q["done"] == 1 and q["lam"] == 4 * lam
        with pytest.raises(eng.CmaesError):
            eng.cmaes_restart(h, 0)
    finally:
        eng.cmaes_destroy(h)


def test_held_then_restarted_descent_matches_oracle_restart():
    """A search that stopped under restart_hold and is restarted by the host
    (the K-Replicated schedule's merge) gets the oracle's restart: lambda
    doubled, the Philox mean of its restart index, sigma0, C = B = I, zero
    paths; and its first generation after the restart matches the oracle's."""
    import paper_2409_11765_gb300 as eng
    from oracle import cmaes
    from paper_2409_11765_gb300 import workloads as W
    from parity_util import oracle_problem, rel
    n, lam = 8, 6
    p = W.make_problem(W.ELLIPSOID, n, SEED, 5, cond=1e2)
    opt = eng.cmaes_default_options(max_restarts=2, ipop_double=1, restart_hold=1, max_iter=5,
                                    box_lo=-3.0, box_hi=3.0)
    h = eng.cmaes_create(n, lam, np.ones(n), 1.0, SEED, opt)
    try:
        eng.cmaes_set_problem(h, 0, p.kind, p.Q, p.lamdiag, p.xstar)
        eng.cmaes_step_batch(h, 8)
        held = eng.cmaes_get_state(h, 0, n)
        assert held["done"] == 2
        eng.cmaes_restart(h, 0)
        g0 = eng.cmaes_get_state(h, 0, n)
        eng.cmaes_step_batch(h, 1)
        g1 = eng.cmaes_get_state(h, 0, n)
    finally:
        eng.cmaes_destroy(h)
    opts = cmaes.Options(max_restarts=2, ipop_double=True, max_iter=5, box_lo=-3.0, box_hi=3.0)
    st = cmaes.State(n, lam, held["sigma"], held["m"].copy(), 1.0, best_f=held["best_f"],
                     best_x=held["best_x"].copy())
    cmaes.restart(st, SEED, 0, opts)
    assert g0["lam"] == st.lam == 2 * lam and g0["restart"] == st.restart == 1 and g0["gen"] == 0
    assert np.abs(g0["m"] - st.m).max() <= 1e-15 * 3.0
    assert g0["sigma"] == st.sigma == 1.0
    assert np.array_equal(g0["C"], np.eye(n)) and np.array_equal(g0["B"], np.eye(n))
    assert not g0["ps"].any() and not g0["pc"].any() and g0["best_f"] == st.best_f
    cmaes.generation(st, SEED, 0, oracle_problem(p), opts)
    for k in ("m", "ps", "pc", "C"):
        assert rel(g1[k], getattr(st, k)) <= 1e-12, k
    assert math.isclose(g1["sigma"], st.sigma, rel_tol=1e-12)


@pytest.mark.parametrize("kind", ["kdistributed", "kreplicated"])
def test_strategies_reach_all_targets_on_a_small_ellipsoid(kind):
    from paper_2409_11765_gb300 import strategies as S
    r = S.run_strategy(kind, "ellipsoid", 6, 6, 1, seed=3, precision=0, max_gens=3000,
                       check_every=5)
    assert all(h is not None for h in r["hits"]), r["hits"]
    t = [h["device_ms"] for h in r["hits"]]
    assert all(b >= a for a, b in zip(t, t[1:]))  # harder targets are hit later
    assert r["best"] < 1e-8 and r["candidates_per_s"] > 0

"""Asynchronous batched ask / tell against the synchronous per-search path:
the searches are independent, so both give bit-identical states."""
import numpy as np
import pytest

from parity_util import SEED, have_gpu

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _handle(prec):
    import paper_2409_11765_gb300 as eng
    from paper_2409_11765_gb300 import workloads as W
    from paper_2409_11765_gb300.external import host_objective
    ns, lams = [12, 7, 33], [10, 9, 40]
    kinds = [W.ELLIPSOID, W.SPHERE, W.RASTRIGIN]
    opt = eng.cmaes_default_options(precision=prec, eig_every=1, max_restarts=0)
    h = eng.cmaes_create_batch(ns, lams, [np.full(n, 0.5) for n in ns], [1.0] * 3, SEED, opt)
    fns = []
    for i, (n, k) in enumerate(zip(ns, kinds)):
        p = W.make_problem(k, n, SEED, 50 + i, cond=1e3)
        eng.cmaes_set_problem(h, i, p.kind, p.Q, p.lamdiag, p.xstar)
        fns.append(host_objective(p.kind, p.Q, p.lamdiag, p.xstar))
    return eng, h, ns, lams, fns


@pytest.mark.parametrize("prec", [0, 1])
def test_async_groups_match_sync_ask_tell(prec):
    from paper_2409_11765_gb300.external import AsyncAskTell, run_sync
    eng, h1, ns, lams, fns = _handle(prec)
    _, h2, _, _, _ = _handle(prec)
    try:
        gens = 6
        c1 = run_sync(h1, ns, fns, gens)
        pipe = AsyncAskTell(h2, ns, lams, [(2, 3), (0, 2)])
        c2 = pipe.run(fns, gens)
        assert c1 == c2 == gens * sum(lams)
        for s, n in enumerate(ns):
            a, b = eng.cmaes_get_state(h1, s, n), eng.cmaes_get_state(h2, s, n)
            for k in ("m", "C", "B", "D", "ps", "pc"):
                assert np.array_equal(a[k], b[k]), (s, k)
            assert a["sigma"] == b["sigma"] and a["gen"] == b["gen"] == gens
            assert a["best_f"] == b["best_f"]
    finally:
        eng.cmaes_destroy(h1)
        eng.cmaes_destroy(h2)


def test_async_argument_checks():
    import paper_2409_11765_gb300 as eng
    eng_, h, ns, lams, fns = _handle(0)
    try:
        buf = np.zeros(12 * 10)
        with pytest.raises(eng.CmaesError):
            eng.cmaes_tell_async(h, 0, 1, [buf.ctypes.data])     # tell without ask
        with pytest.raises(eng.CmaesError):
            eng.cmaes_ask_async(h, 2, 1, [buf.ctypes.data], buf.ctypes.data)  # empty range
    finally:
        eng.cmaes_destroy(h)


def test_async_groups_follow_the_oracle():
    """The asynchronous path against the oracle: every search starts from a
    teacher-forced state with distinct eigenvalues, the host evaluates f with
    the oracle's objectives, and after each generation every search's state
    matches the oracle's generation fed the same points' values."""
    import paper_2409_11765_gb300 as eng
    from oracle import cmaes, objectives
    from paper_2409_11765_gb300 import workloads as W
    from paper_2409_11765_gb300.external import AsyncAskTell
    from parity_util import oracle_state, rel, state_dict
    ns, lams = [12, 7, 33], [10, 9, 40]
    kinds = [W.ELLIPSOID, W.SPHERE, W.RASTRIGIN]
    opt = eng.cmaes_default_options(precision=0, eig_every=1, max_restarts=0)
    states = [W.random_state(n, SEED, 600 + i, cond=1e2) for i, n in enumerate(ns)]
    probs = [W.make_problem(k, n, SEED, 50 + i, cond=1e3) for i, (n, k) in enumerate(zip(ns, kinds))]
    h = eng.cmaes_create_batch(ns, lams, [d["m"] for d in states], [1.0] * 3, SEED, opt)
    fns = [lambda X, p=p: objectives.evaluate(p.kind, X, p.Q, p.lamdiag, p.xstar) for p in probs]
    orc = [oracle_state(d, n, lam, 1.0, gen=1) for d, n, lam in zip(states, ns, lams)]
    opts = cmaes.Options(eig_every=1, max_restarts=0)
    try:
        for i, p in enumerate(probs):
            eng.cmaes_set_problem(h, i, p.kind, p.Q, p.lamdiag, p.xstar)
            eng.cmaes_set_state(h, i, state_dict(states[i], ns[i], lams[i], gen=1))
        pipe = AsyncAskTell(h, ns, lams, [(2, 3), (0, 2)])
        for g in range(4):
            pipe.run(fns, 1)
            for i in range(3):
                cmaes.generation(orc[i], SEED, i, cmaes.Problem(probs[i].kind, probs[i].xstar,
                                                                probs[i].Q, probs[i].lamdiag), opts)
                s = eng.cmaes_get_state(h, i, ns[i])
                tol = 1e-12 * 10 ** (g / 5)
                assert s["gen"] == orc[i].gen
                assert rel(s["m"], orc[i].m) < tol, (g, i, rel(s["m"], orc[i].m))
                assert rel(s["C"], orc[i].C) < tol, (g, i)
                assert abs(s["sigma"] / orc[i].sigma - 1) < tol
                assert abs(s["best_f"] - orc[i].best_f) <= tol * max(1.0, abs(orc[i].best_f))
    finally:
        eng.cmaes_destroy(h)

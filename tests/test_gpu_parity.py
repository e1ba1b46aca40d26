"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Every test feeds the same seeded inputs and the same state to both sides; the
random draws are Philox4x32-10 counters implemented independently on each side.
FP64 path tolerance: 1e-12 normwise relative for every state quantity, rank
order bit-exact.
"""
import math

import numpy as np
import pytest

from parity_util import (SEED, TOL_FP64, check_generation, have_gpu, oracle_problem, rel,
                         teacher_forced)

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _states(ns, stream0=0, cond=1e3):
    from paper_2409_11765_gb300 import workloads as W
    return [W.random_state(n, SEED, stream0 + i, cond=cond) for i, n in enumerate(ns)]


@pytest.mark.parametrize("n,lam,kind", [
    (10, 10, 1),      # the small ellipsoid
    (1, 2, 3),        # degenerate: n = 1, lambda = 2
    (2, 6, 2),
    (7, 9, 1),        # odd n: the Jacobi dummy index
    (65, 130, 2),     # ragged 64-tiles in both GEMM dimensions
    (100, 17, 2),     # Rastrigin n = 100, lambda0 = 17
    (100, 1088, 1),   # several rank / recombination chunks
    (33, 20, 1),      # smallest cluster-Jacobi size: two CTAs of the cluster idle
    (130, 40, 1),     # cluster Jacobi
    (159, 30, 2),     # refined route, odd n: the padding pair of the FP32 Jacobi
    (160, 40, 1),     # largest refined-route size: four 2 x 2 blocks per FP32 Jacobi thread
    (161, 32, 2),     # smallest size of the many-CTA FP32 Jacobi, odd n
    (256, 30, 2),     # largest cluster-Jacobi size (cleanup of the many-CTA route)
    (300, 40, 1),     # global-memory Jacobi (cleanup of the many-CTA route)
])
def test_teacher_forced_generation(n, lam, kind):
    gpu, ora = teacher_forced([n], [lam], [kind], _states([n]), eig_every=1)
    check_generation(gpu, ora)


def test_generation_without_eig_keeps_B_D():
    gpu, ora = teacher_forced([20], [12], [1], _states([20], 3), eig_every=1000)
    check_generation(gpu, ora, eig=False)


def test_batch_of_uneven_searches():
    ns, lams, kinds = [10, 33, 100, 5], [10, 70, 17, 300], [1, 2, 2, 3]
    states = _states(ns, 10)
    for s in range(len(ns)):
        gpu, ora = teacher_forced(ns, lams, kinds, states, search=s, eig_every=1)
        check_generation(gpu, ora)


def test_batch_of_uneven_large_searches():
    """Several searches on the many-CTA FP32 Jacobi (different n, so different
    step counts per sweep) share its launches with a one-CTA-route search."""
    ns, lams, kinds = [40, 170, 261], [20, 30, 24], [1, 2, 1]
    states = _states(ns, 40)
    for s in range(len(ns)):
        gpu, ora = teacher_forced(ns, lams, kinds, states, search=s, eig_every=1)
        check_generation(gpu, ora)


def test_batch_invariance_bitwise():
    """A search gives bit-identical results alone and inside a batch."""
    import paper_2409_11765_gb300 as eng
    from paper_2409_11765_gb300 import workloads as W
    ns, lams = [12, 40, 12], [8, 50, 8]
    probs = [W.make_problem(1, n, SEED, 90 + i) for i, n in enumerate(ns)]
    x0s = [W.start_point(n, -4, 4, SEED, 90 + i) for i, n in enumerate(ns)]
    opt = eng.cmaes_default_options(max_restarts=2)

    def run(idx):
        h = eng.cmaes_create_batch([ns[i] for i in idx], [lams[i] for i in idx],
                                   [x0s[i] for i in idx], [1.0] * len(idx), SEED, opt)
        try:
            for j, i in enumerate(idx):
                eng.cmaes_set_problem(h, j, 1, probs[i].Q, probs[i].lamdiag, probs[i].xstar)
            eng.cmaes_step_batch(h, 25)
            return eng.cmaes_get_state(h, len(idx) - 1, ns[idx[-1]])
        finally:
            eng.cmaes_destroy(h)

    # search 2 runs as the third of three, and as the third with another
    # neighbour set: the Philox stream index is the position in the batch
    a = run([0, 1, 2])
    b = run([1, 0, 2])
    for k in ("m", "C", "B", "D", "ps", "pc"):
        assert np.array_equal(a[k], b[k]), k
    assert a["sigma"] == b["sigma"]


def test_ask_tell_ranks_ties_and_nan_bit_exact():
    """External f with ties, NaN and infinities: the order is bit-exact."""
    import paper_2409_11765_gb300 as eng
    from oracle import cmaes
    from paper_2409_11765_gb300 import workloads as W
    n, lam = 6, 24
    d = W.random_state(n, SEED, 40)
    h = eng.cmaes_create(n, lam, d["m"], 1.0, SEED, eng.cmaes_default_options(eig_every=1))
    try:
        eng.cmaes_set_state(h, 0, dict(n=n, lam=lam, sigma=d["sigma"], m=d["m"], ps=d["ps"],
                                       pc=d["pc"], C=d["C"], B=d["B"], D=d["D"], gen=2))
        X = eng.cmaes_ask(h, 0, n)
        with pytest.raises(eng.CmaesError):
            eng.cmaes_ask(h, 0, n)          # ask twice: ESTATE
        vals = np.array([3.0, 1.0, np.nan, 1.0, -np.inf, 0.0, -0.0, 1.0, np.inf, 2.0, np.nan, 0.0])
        f = np.resize(vals, lam)
        eng.cmaes_tell(h, 0, f)
        with pytest.raises(eng.CmaesError):
            eng.cmaes_tell(h, 0, f)         # tell without ask: ESTATE
        _, _, order = eng.cmaes_get_generation(h, 0, n)
        g = eng.cmaes_get_state(h, 0, n)
    finally:
        eng.cmaes_destroy(h)
    st = cmaes.State(n, lam, d["sigma"], d["m"].copy(), 1.0, d["ps"].copy(), d["pc"].copy(),
                     d["C"].copy(), d["B"].copy(), d["D"].copy(), gen=2)
    from oracle import philox
    Z = philox.normals(SEED, 0, 0, 2, n, lam)
    Y, Xo = cmaes.sample(st, Z)
    assert rel(X, Xo) <= TOL_FP64
    rec = cmaes.generation(st, SEED, 0, None, cmaes.Options(eig_every=1), Z=Z, f=f)
    assert np.array_equal(order, rec["order"])
    assert rel(g["m"], st.m) <= TOL_FP64 and rel(g["C"], st.C) <= TOL_FP64


def test_forced_restart_and_ipop_doubling():
    import paper_2409_11765_gb300 as eng
    from oracle import philox
    n, lam = 9, 8
    opt = eng.cmaes_default_options(max_restarts=3, box_lo=-5.0, box_hi=5.0)
    h = eng.cmaes_create(n, lam, np.zeros(n), 2.5, SEED, opt)
    try:
        eng.cmaes_restart(h, 0)
        q = eng.cmaes_query(h, 0)
        g = eng.cmaes_get_state(h, 0, n)
    finally:
        eng.cmaes_destroy(h)
    assert q["lam"] == 16 and q["restart"] == 1 and q["gen"] == 0
    m_ref = philox.restart_mean(SEED, 0, 1, n, -5.0, 5.0)
    assert np.abs(g["m"] - m_ref).max() <= 1e-15 * 5.0
    assert np.array_equal(g["C"], np.eye(n)) and g["sigma"] == 2.5


def test_state_roundtrip():
    import paper_2409_11765_gb300 as eng
    from paper_2409_11765_gb300 import workloads as W
    n, lam = 11, 14
    d = W.random_state(n, SEED, 41)
    h = eng.cmaes_create(n, lam, d["m"], 1.0, SEED)
    try:
        hist = np.linspace(1, 2, 7)
        eng.cmaes_set_state(h, 0, dict(n=n, lam=lam, sigma=0.3, m=d["m"], ps=d["ps"], pc=d["pc"],
                                       C=d["C"], B=d["B"], D=d["D"], gen=5, restart=0,
                                       best_f=1.5, best_x=d["m"], hist=hist))
        g = eng.cmaes_get_state(h, 0, n)
    finally:
        eng.cmaes_destroy(h)
    for k in ("m", "ps", "pc", "C", "B", "D"):
        assert np.array_equal(g[k], d[k]), k
    assert g["gen"] == 5 and g["sigma"] == 0.3 and g["best_f"] == 1.5
    assert np.array_equal(g["hist"], hist)


def test_small_ellipsoid_reaches_target():
    """Plain CMA-ES, n=10, lambda=10, rotated ellipsoid cond 1e6, from the
    configuration's own start: f < 1e-10 within 2000 generations, confirmed by
    an FP64 re-evaluation of the returned point. (From C = I the first updates
    leave C with a repeated eigenvalue, whose eigenvectors any solver may pick
    differently, so this run is compared by outcome, not step by step.)"""
    import paper_2409_11765_gb300 as eng
    from oracle import objectives
    from paper_2409_11765_gb300 import workloads as W
    wl = W.ellipsoid_n10()
    s = wl.searches[0]
    opt = eng.cmaes_default_options(f_target=wl.f_target, max_restarts=0, box_lo=-4.0, box_hi=4.0)
    h = eng.cmaes_create(s.n, s.lam, s.x0, s.sigma0, SEED, opt)
    try:
        p = s.problem
        eng.cmaes_set_problem(h, 0, p.kind, p.Q, p.lamdiag, p.xstar)
        eng.cmaes_step_batch(h, wl.generations)
        q = eng.cmaes_query(h, 0)
        x, fbest = eng.cmaes_best(h, 0, s.n)
    finally:
        eng.cmaes_destroy(h)
    assert q["done"] == 1 and q["flags"] & 1
    assert fbest < 1e-10
    f_re = objectives.evaluate(p.kind, x[:, None], p.Q, p.lamdiag, p.xstar)[0]
    assert f_re < 1e-10 and math.isclose(f_re, fbest, rel_tol=1e-6, abs_tol=1e-14)


def test_full_size_rastrigin_n100_lambda8704_sampled():
    """Full size of the largest IPOP level (n=100, lambda=8704) in the launch
    configuration the benchmark times: the whole generation against the oracle
    (cheap here), with the sample columns also recomputed one by one."""
    n, lam = 100, 8704
    states = _states([n], 60)
    gpu, ora = teacher_forced([n], [lam], [2], states, eig_every=1, sigma0=2.5)
    check_generation(gpu, ora)
    d = states[0]
    from oracle import philox
    idx = [0, 1, 4095, 8703]
    for k in idx:
        z = philox.normals(SEED, 0, 0, 3, n, k + 1)[:, k]
        xk = d["m"] + d["sigma"] * (d["B"] @ (d["D"] * z))
        assert rel(gpu["X"][:, k], xk) <= TOL_FP64


def test_kdistributed_levels_full_batch():
    """The benchmark's batch: ten Rastrigin levels lambda = 17 * 2^k side by
    side; every search's generation matches the oracle."""
    ns = [100] * 10
    lams = [17 << k for k in range(10)]
    kinds = [2] * 10
    states = _states(ns, 70)
    for s in (0, 5, 9):
        gpu, ora = teacher_forced(ns, lams, kinds, states, search=s, eig_every=1, sigma0=2.5,
                                  opt_over=dict(ipop_double=False, max_restarts=255,
                                                box_lo=-5.0, box_hi=5.0))
        check_generation(gpu, ora)


@pytest.mark.parametrize("n,lam,kind,gens", [(10, 10, 1, 25), (30, 20, 2, 20), (100, 17, 2, 10),
                                             (100, 2176, 2, 6)])
def test_trajectory_follows_oracle(n, lam, kind, gens):
    """Many generations in a row, each with a warm-started eigendecomposition,
    from a state whose eigenvalues are distinct: with the canonical eigenbasis
    the GPU and oracle trajectories stay together (the dynamics amplify
    rounding differences only slowly)."""
    import paper_2409_11765_gb300 as eng
    from oracle import cmaes
    from paper_2409_11765_gb300 import workloads as W
    from parity_util import oracle_state, state_dict
    p = W.make_problem(kind, n, SEED, 300 + n)
    d = W.random_state(n, SEED, 300 + n, cond=1e2)
    d["sigma"] = 1.0
    opt = eng.cmaes_default_options(eig_every=1, max_restarts=0)
    h = eng.cmaes_create(n, lam, d["m"], 2.0, SEED, opt)
    st = oracle_state(d, n, lam, 2.0, gen=1)
    opts = cmaes.Options(eig_every=1, max_restarts=0)
    try:
        eng.cmaes_set_problem(h, 0, p.kind, p.Q, p.lamdiag, p.xstar)
        eng.cmaes_set_state(h, 0, state_dict(d, n, lam, gen=1))
        for g in range(gens):
            eng.cmaes_step_batch(h, 1)
            cmaes.generation(st, SEED, 0, oracle_problem(p), opts)
            s = eng.cmaes_get_state(h, 0, n)
            tol = 1e-12 * 10 ** (g / 5)
            assert rel(s["m"], st.m) < tol, (g, rel(s["m"], st.m))
            assert rel(s["C"], st.C) < tol, (g, rel(s["C"], st.C))
            assert abs(s["sigma"] / st.sigma - 1) < tol
    finally:
        eng.cmaes_destroy(h)

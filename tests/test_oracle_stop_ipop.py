"""Pins for the stop tests, the IPOP restart (Algorithm 2) and end to end runs."""
import math

import numpy as np
import pytest

from oracle import cmaes, philox
from oracle.params import Params
from paper_2409_11765_gb300 import workloads as W


def _fresh(n=4, lam=8, sigma=1.0):
    return cmaes.State(n, lam, sigma, np.zeros(n), sigma)


def test_each_stop_flag():
    opts = cmaes.Options(f_target=1e-8)
    n, lam = 4, 8
    p = Params(n, lam)
    st = _fresh(n, lam)
    assert cmaes.stop_flags(st, p, opts) == 0
    st.best_f = 1e-9
    assert cmaes.stop_flags(st, p, opts) == cmaes.STOP_FTARGET
    st = _fresh(n, lam)
    st.gen = p.max_iter
    assert cmaes.stop_flags(st, p, opts) & cmaes.STOP_MAXITER
    st = _fresh(n, lam)
    st.hist = [1.0] * p.hist_len
    assert cmaes.stop_flags(st, p, opts) == cmaes.STOP_TOLHISTFUN
    st.hist[-1] = 1.0 + 1e-9
    assert cmaes.stop_flags(st, p, opts) == 0
    st = _fresh(n, lam)
    st.sigma = 1e-13
    f = cmaes.stop_flags(st, p, opts)
    assert f & cmaes.STOP_TOLX
    st = _fresh(n, lam)
    st.D = np.array([1.0, 1.0, 1.0, 1e-8])
    assert cmaes.stop_flags(st, p, opts) == cmaes.STOP_CONDITIONCOV
    st = _fresh(n, lam)
    st.m = np.full(n, 1e20)
    assert cmaes.stop_flags(st, p, opts) & cmaes.STOP_NOEFFECTAXIS
    assert cmaes.stop_flags(st, p, opts) & cmaes.STOP_NOEFFECTCOORD
    st = _fresh(n, lam)
    st.m = np.array([1e20, 0.0, 0.0, 0.0])
    st.gen = 1                        # NoEffectAxis probes axis gen mod n = 1
    assert cmaes.stop_flags(st, p, opts) == cmaes.STOP_NOEFFECTCOORD
    st = _fresh(n, lam)
    st.sigma = math.nan
    assert cmaes.stop_flags(st, p, opts) & cmaes.STOP_NONFINITE


def test_restart_doubles_lambda_and_resets():
    opts = cmaes.Options(box_lo=-5.0, box_hi=5.0, max_restarts=3)
    st = _fresh(6, 10, 2.5)
    st.gen, st.sigma, st.best_f = 40, 1e-3, 0.5
    st.C = 2 * np.eye(6)
    st.hist = [1.0, 2.0]
    cmaes.restart(st, 77, 3, opts)
    assert st.lam == 20 and st.restart == 1 and st.gen == 0
    assert st.sigma == 2.5 and np.array_equal(st.C, np.eye(6)) and st.hist == []
    assert np.array_equal(st.m, philox.restart_mean(77, 3, 1, 6, -5.0, 5.0))
    assert st.best_f == 0.5           # the best point is kept over all descents
    opts.ipop_double = False
    cmaes.restart(st, 77, 3, opts)
    assert st.lam == 20 and st.restart == 2


def test_ipop_lambda_sequence_and_final_stop():
    """Algorithm 2: K = 1, 2, 4, ... up to K_max, then the search ends."""
    opts = cmaes.Options(max_restarts=3, max_iter=3)
    pr = cmaes.Problem(W.SPHERE, np.zeros(3))
    st = cmaes.State(3, 5, 1.0, np.ones(3), 1.0)
    lams = []
    while not st.done:
        lams.append(st.lam)
        cmaes.generation(st, 1, 0, pr, opts)
    assert sorted(set(lams)) == [5, 10, 20, 40]
    assert st.restart == 3 and st.flags & cmaes.STOP_MAXITER


def test_config0_reaches_target():
    """Plain CMA-ES on the n=10 rotated ellipsoid (cond 1e6) reaches 1e-10."""
    wl = W.ellipsoid_n10()
    s = wl.searches[0]
    st = cmaes.State(s.n, s.lam, s.sigma0, s.x0.copy(), s.sigma0)
    pr = cmaes.Problem(s.problem.kind, s.problem.xstar, s.problem.Q, s.problem.lamdiag)
    opts = cmaes.Options(f_target=wl.f_target, box_lo=wl.box_lo, box_hi=wl.box_hi,
                         max_restarts=0, ipop_double=False)
    g = cmaes.run(st, W.SEED, 0, pr, opts, wl.generations)
    assert st.best_f < 1e-10 and st.flags & cmaes.STOP_FTARGET
    assert g < wl.generations
    # C stays symmetric positive definite and B orthonormal along the way
    assert np.allclose(st.C, st.C.T, atol=0)
    assert np.linalg.eigvalsh(st.C).min() > 0
    assert np.abs(st.B.T @ st.B - np.eye(s.n)).max() < 1e-13 * s.n


def test_invariants_along_trajectory():
    n, lam = 8, 12
    pr = cmaes.Problem(W.ELLIPSOID, np.zeros(n), W.haar_orthogonal(n, W.rng_for(1, 9)),
                       W.ellipsoid_diag(n, 1e3))
    st = cmaes.State(n, lam, 1.0, np.ones(n), 1.0)
    opts = cmaes.Options(max_restarts=0)
    for _ in range(60):
        rec = cmaes.generation(st, 3, 0, pr, opts)
        # the mean moved by the sampling identity m' - m = sigma B D <z>_w
        if rec["eig"]:
            assert np.linalg.norm((st.B * st.D ** 2) @ st.B.T - st.C) <= 1e-12 * np.linalg.norm(st.C)
        assert np.abs(st.B.T @ st.B - np.eye(n)).max() <= 1e-13 * n
        assert np.linalg.eigvalsh(0.5 * (st.C + st.C.T)).min() > 0


def test_mean_shift_equals_sampling_identity():
    n, lam = 5, 9
    pr = cmaes.Problem(W.SPHERE, np.zeros(n))
    st = cmaes.State(n, lam, 0.7, np.ones(n), 0.7)
    d = W.random_state(n, 2, 3)
    st.B, st.D, st.C = d["B"], d["D"], d["C"]
    B, D, sigma, m0 = st.B.copy(), st.D.copy(), st.sigma, st.m.copy()
    rec = cmaes.generation(st, 3, 0, pr, cmaes.Options(eig_every=1000))
    assert np.allclose(st.m - m0, sigma * (B @ (D * rec["zw"])), rtol=1e-13, atol=1e-15)

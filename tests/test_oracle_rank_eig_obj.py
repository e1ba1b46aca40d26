"""Pins for ranking, the eigendecomposition step and the objectives."""
import itertools
import math

import numpy as np
import pytest

from oracle import cmaes, objectives
from paper_2409_11765_gb300 import workloads as W


def _brute_rank(f):
    """All-pairs: candidate k's rank counts j with (key_j, j) < (key_k, k)."""
    key = [math.inf if math.isnan(v) else v for v in f]
    lam = len(f)
    order = [None] * lam
    for k in range(lam):
        r = sum(1 for j in range(lam) if (key[j] < key[k]) or (key[j] == key[k] and j < k))
        order[r] = k
    return order


@pytest.mark.parametrize("lam", [1, 2, 3, 5, 8])
def test_rank_brute_force_with_ties(lam):
    vals = [0.0, -0.0, 1.0, -1.0, math.nan, math.inf, -math.inf, 2.0]
    rng = np.random.default_rng(lam)
    for _ in range(300):
        f = [vals[i] for i in rng.integers(0, len(vals), size=lam)]
        assert list(cmaes.rank_order(np.array(f))) == _brute_rank(f)


def test_rank_constant_is_identity():
    # sigma -> 0 makes f constant: the order is the index order
    assert list(cmaes.rank_order(np.full(9, 3.25))) == list(range(9))
    assert list(cmaes.rank_order(np.full(4, math.nan))) == [0, 1, 2, 3]


def test_rank_all_permutations_small():
    for perm in itertools.permutations(range(5)):
        f = np.array(perm, dtype=float)
        assert list(cmaes.rank_order(f)) == list(np.argsort(f))


@pytest.mark.parametrize("n", [2, 5, 30])
def test_eig_step_reconstructs(n):
    d = W.random_state(n, 21, n, cond=1e6)
    st = cmaes.State(n, 10, 1.0, np.zeros(n), 1.0, C=d["C"].copy())
    cmaes.eig_step(st)
    B, D = st.B, st.D
    assert np.abs(B.T @ B - np.eye(n)).max() <= 1e-13 * n
    rec = (B * D ** 2) @ B.T
    assert np.linalg.norm(rec - st.C) <= 1e-12 * np.linalg.norm(st.C)
    assert np.allclose(np.sort(D ** 2), np.sort(d["D"] ** 2), rtol=1e-9)


def test_eig_2x2_closed_form():
    a, b, c = 3.0, 0.75, 0.5
    st = cmaes.State(2, 4, 1.0, np.zeros(2), 1.0, C=np.array([[a, b], [b, c]]))
    cmaes.eig_step(st)
    tr, det = a + c, a * c - b * b
    disc = math.sqrt(tr * tr / 4 - det)
    assert np.allclose(np.sort(st.D ** 2), [tr / 2 - disc, tr / 2 + disc], rtol=1e-15)


def test_eig_pd_guard():
    C = np.diag([4.0, 1.0, -1e-3])
    st = cmaes.State(3, 4, 1.0, np.zeros(3), 1.0, C=C)
    cmaes.eig_step(st)
    floor = 4.0 * (1 + 0) * cmaes.PD_FLOOR
    lifted = 4.0 * cmaes.PD_FLOOR + 1e-3
    assert np.all(st.D ** 2 > 0)
    assert math.isclose(min(st.D ** 2), 4.0 * cmaes.PD_FLOOR, rel_tol=1e-6) or min(st.D ** 2) >= floor
    assert np.allclose(np.diag(st.C), [4.0 + lifted, 1.0 + lifted, -1e-3 + lifted])


def test_haar_orthogonal():
    rng = W.rng_for(1, 2)
    for n in (1, 2, 10, 100):
        Q = W.haar_orthogonal(n, rng)
        assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-14 * max(n, 10)
        assert math.isclose(abs(np.linalg.det(Q)), 1.0, rel_tol=1e-12)


def test_objectives_special_points():
    n = 12
    pe = W.make_problem(W.ELLIPSOID, n, 5, 0, cond=1e6)
    pr = W.make_problem(W.RASTRIGIN, n, 5, 1)
    ps = W.make_problem(W.SPHERE, n, 5, 2)
    for p in (pe, pr, ps):
        X = p.xstar[:, None]
        assert objectives.evaluate(p.kind, X, p.Q, p.lamdiag, p.xstar)[0] == pytest.approx(0.0, abs=1e-12)
    # ellipsoid with Q = I is the weighted separable sum
    X = np.random.default_rng(0).standard_normal((n, 5))
    f = objectives.ellipsoid(X, np.eye(n), pe.lamdiag, pe.xstar)
    expect = [(pe.lamdiag * (X[:, k] - pe.xstar) ** 2).sum() for k in range(5)]
    assert np.allclose(f, expect, rtol=1e-14)
    # Rastrigin at integer offsets in the rotated frame is sum u^2
    u = np.array([1.0, -2.0] + [0.0] * (n - 2))
    x = pr.xstar + pr.Q.T @ u
    assert objectives.rastrigin(x[:, None], pr.Q, pr.xstar)[0] == pytest.approx(5.0, abs=1e-10)
    # ellipsoid spectrum runs from 1 to cond
    assert pe.lamdiag[0] == 1.0 and math.isclose(pe.lamdiag[-1], 1e6, rel_tol=1e-14)


def test_canonical_eigenbasis_is_unique():
    """Any orthonormal eigenbasis (columns permuted, signs flipped) maps to the
    same representative: ascending eigenvalues, largest entry positive."""
    n = 8
    d = W.random_state(n, 23, 1, cond=1e4)
    st = cmaes.State(n, 10, 1.0, np.zeros(n), 1.0, C=d["C"].copy())
    cmaes.eig_step(st)
    assert np.all(np.diff(st.D) > 0)
    B = st.B
    idx = np.argmax(np.abs(B), axis=0)
    assert np.all(B[idx, np.arange(n)] > 0)
    rng = np.random.default_rng(0)
    perm = rng.permutation(n)
    flipped = (d["B"] * rng.choice([-1.0, 1.0], size=n))[:, perm]
    order = np.argsort(d["D"][perm])
    again = cmaes.canonical_basis(flipped[:, order])
    assert np.allclose(again, B, atol=1e-10)

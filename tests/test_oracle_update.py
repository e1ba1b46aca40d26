"""Pins for one oracle generation (Eq. (1), Eq. (2)/(3) and the update)."""
import math

import numpy as np
import pytest
from scipy.linalg import fractional_matrix_power

from oracle import cmaes
from oracle.params import Params
from paper_2409_11765_gb300 import workloads as W


def _state_from(d, n, lam, sigma0=1.0):
    return cmaes.State(n, lam, d["sigma"], d["m"].copy(), sigma0, d["ps"].copy(),
                       d["pc"].copy(), d["C"].copy(), d["B"].copy(), d["D"].copy())


def test_hand_worked_n2_generation():
    """n=2, lambda=6, m=0, sigma=1, C=B=D=I, p=0, g=0, f=||x-(1,0)||^2 and six
    chosen z. The tie f=2 between candidates 1 and 3 decides the selection by
    index. Expected values re-derived here with scalar arithmetic."""
    st = cmaes.State(2, 6, 1.0, np.zeros(2), 1.0)
    p = Params(2, 6)
    zs = [(1, 0), (0, 1), (-1, 0), (0, -1), (0.5, 0.5), (-0.5, 0.5)]
    Z = np.array(zs, dtype=float).T
    Y, X = cmaes.sample(st, Z)
    f = np.array([(x - 1.0) ** 2 + y ** 2 for x, y in zs])
    rec = cmaes.update(st, p, Z, Y, X, f)
    assert list(rec["order"]) == [0, 4, 1, 3, 5, 2]
    w = p.weights
    sel = [zs[0], zs[4], zs[1]]
    yw = [sum(w[i] * sel[i][c] for i in range(3)) for c in range(2)]
    assert np.allclose(st.m, yw, rtol=0, atol=1e-15)
    coef = math.sqrt(p.cs * (2 - p.cs) * p.mueff)
    ps = [coef * yw[0], coef * yw[1]]
    assert np.allclose(st.ps, ps, rtol=0, atol=1e-15)
    psn = math.hypot(*ps)
    assert rec["hsig"] == 1.0
    pc = [math.sqrt(p.cc * (2 - p.cc) * p.mueff) * v for v in yw]
    assert np.allclose(st.pc, pc, rtol=0, atol=1e-15)
    a = 1 - p.c1 - p.cmu
    C = [[a + p.c1 * pc[0] * pc[0] + p.cmu * sum(w[i] * sel[i][0] * sel[i][0] for i in range(3)),
          p.c1 * pc[0] * pc[1] + p.cmu * sum(w[i] * sel[i][0] * sel[i][1] for i in range(3))],
         [0.0, a + p.c1 * pc[1] * pc[1] + p.cmu * sum(w[i] * sel[i][1] * sel[i][1] for i in range(3))]]
    C[1][0] = C[0][1]
    assert np.allclose(st.C, C, rtol=0, atol=1e-15)
    sig = math.exp((p.cs / p.ds) * (psn / p.chin - 1))
    assert math.isclose(st.sigma, sig, rel_tol=1e-15)
    # the same to 12 digits (hand derivation)
    assert np.allclose(st.m, [0.779327699960, 0.220672300040], atol=5e-13)
    assert np.allclose(st.ps, [0.924237578030, 0.261704584782], atol=5e-13)
    assert abs(psn - 0.960575031082) < 5e-13
    assert np.allclose(st.pc, [1.028789261228, 0.291309153445], atol=5e-13)
    assert np.allclose(st.C, [[0.992158215257, 0.050513757779],
                              [0.050513757779, 0.809114961922]], atol=5e-13)
    tr, det = st.C[0, 0] + st.C[1, 1], st.C[0, 0] * st.C[1, 1] - st.C[0, 1] ** 2
    ev = sorted([tr / 2 - math.sqrt(tr * tr / 4 - det), tr / 2 + math.sqrt(tr * tr / 4 - det)])
    assert abs(ev[0] - 0.796100241452) < 5e-13 and abs(ev[1] - 1.005172935727) < 5e-13
    assert abs(st.sigma - 0.930302115988) < 5e-13
    assert st.best_f == 0.0 and np.array_equal(st.best_x, [1.0, 0.0])
    assert st.gen == 1


@pytest.mark.parametrize("n,lam", [(5, 12), (13, 40)])
def test_eq2_equals_eq3(n, lam):
    """The rank-mu form applied by the oracle equals Eq. (2) written point by
    point with the weights spread over all lambda ranks (zero beyond mu)."""
    d = W.random_state(n, 11, n)
    d["ps"] = d["ps"] * 1e-3            # short path: h_sigma = 1, the case of Eq. (2)
    st = _state_from(d, n, lam)
    C0, pc0 = st.C.copy(), st.pc.copy()
    p = Params(n, lam)
    rng = np.random.default_rng(3)
    Z = rng.standard_normal((n, lam))
    Y, X = cmaes.sample(st, Z)
    f = rng.standard_normal(lam)
    rec = cmaes.update(st, p, Z, Y, X, f)
    assert rec["hsig"] == 1.0
    rank = np.empty(lam, dtype=int)
    rank[rec["order"]] = np.arange(lam)
    w_rk = np.zeros(lam)
    w_rk[:p.mu] = p.weights
    Ceq2 = C0.copy()
    for i in range(lam):
        y = Y[:, i]
        Ceq2 += p.cmu * w_rk[rank[i]] * (np.outer(y, y) - C0)
    pc = st.pc
    Ceq2 += p.c1 * (np.outer(pc, pc) - C0)
    assert np.linalg.norm(st.C - Ceq2) <= 1e-13 * np.linalg.norm(Ceq2)
    # and the paths use the new p_c (Eq. (3) with A = [y_i], B = [w y_i^T])
    assert not np.allclose(pc, pc0)


def test_sampling_gemm_equals_columnwise():
    n, lam = 7, 9
    d = W.random_state(n, 4, 1)
    st = _state_from(d, n, lam)
    Z = np.random.default_rng(0).standard_normal((n, lam))
    Y, X = cmaes.sample(st, Z)
    for k in range(lam):
        yk = np.zeros(n)
        for i in range(n):
            for j in range(n):
                yk[i] += st.B[i, j] * st.D[j] * Z[j, k]
        assert np.allclose(Y[:, k], yk, rtol=1e-14, atol=1e-14)
        assert np.allclose(X[:, k], st.m + st.sigma * yk, rtol=1e-14, atol=1e-14)


def test_psigma_is_inverse_sqrt_of_C():
    """B <z>_w = C^(-1/2) <y>_w when C = B D^2 B^T."""
    n, lam = 9, 20
    d = W.random_state(n, 8, 2)
    st = _state_from(d, n, lam)
    C = (st.B * st.D ** 2) @ st.B.T
    st.C = C
    ps0 = st.ps.copy()
    p = Params(n, lam)
    Z = np.random.default_rng(1).standard_normal((n, lam))
    Y, X = cmaes.sample(st, Z)
    rec = cmaes.update(st, p, Z, Y, X, np.arange(lam, dtype=float))
    coef = math.sqrt(p.cs * (2 - p.cs) * p.mueff)
    Cm12 = np.real(fractional_matrix_power(C, -0.5))
    expect = (1 - p.cs) * ps0 + coef * (Cm12 @ rec["yw"])
    assert np.allclose(st.ps, expect, rtol=1e-10, atol=1e-12)
    # the mean moved by sigma <y>_w, with <y>_w the weighted best steps
    assert np.allclose(rec["yw"], Y[:, :p.mu] @ p.weights, rtol=1e-14, atol=1e-15)


def test_sigma_fixed_point_and_direction():
    n, lam = 6, 10
    p = Params(n, lam)
    # a path of exactly the expected length leaves sigma unchanged
    st = cmaes.State(n, lam, 0.3, np.zeros(n), 0.3)
    Z = np.zeros((n, lam))
    Y, X = cmaes.sample(st, Z)
    target = np.zeros(n)
    target[0] = p.chin / (1 - p.cs)
    st.ps = target
    cmaes.update(st, p, Z, Y, X, np.arange(lam, dtype=float))
    assert math.isclose(st.sigma, 0.3, rel_tol=1e-14)
    # a long path increases it, a zero path decreases it
    st = cmaes.State(n, lam, 0.3, np.zeros(n), 0.3)
    st.ps = 3 * target
    cmaes.update(st, p, Z, Y, X, np.arange(lam, dtype=float))
    assert st.sigma > 0.3
    st = cmaes.State(n, lam, 0.3, np.zeros(n), 0.3)
    cmaes.update(st, p, Z, Y, X, np.arange(lam, dtype=float))
    assert st.sigma < 0.3


def test_hsig_stall():
    """A long p_sigma stalls p_c and keeps the c1 cc (2 - cc) share of C."""
    n, lam = 4, 8
    p = Params(n, lam)
    st = cmaes.State(n, lam, 1.0, np.zeros(n), 1.0)
    st.ps = np.full(n, 50.0)
    st.pc = np.ones(n)
    Z = np.random.default_rng(2).standard_normal((n, lam))
    Y, X = cmaes.sample(st, Z)
    rec = cmaes.update(st, p, Z, Y, X, np.arange(lam, dtype=float))
    assert rec["hsig"] == 0.0
    assert np.allclose(st.pc, (1 - p.cc) * np.ones(n), rtol=1e-15)
    sel = rec["order"][:p.mu]
    rank_mu = (Y[:, sel] * p.weights) @ Y[:, sel].T
    expect = ((1 - p.c1 - p.cmu + p.c1 * p.cc * (2 - p.cc)) * np.eye(n)
              + p.c1 * np.outer(st.pc, st.pc) + p.cmu * rank_mu)
    assert np.allclose(st.C, expect, rtol=1e-14, atol=1e-15)


def test_sphere_expected_value_from_optimum():
    """Separable sphere sampled from m = x* with C = I: E[f] = sigma^2 n."""
    from oracle import philox, objectives
    n, lam, sigma = 50, 4000, 0.2
    xstar = np.linspace(-1, 1, n)
    st = cmaes.State(n, lam, sigma, xstar.copy(), sigma)
    Z = philox.normals(9, 0, 0, 0, n, lam)
    Y, X = cmaes.sample(st, Z)
    f = objectives.sphere(X, xstar)
    # f / sigma^2 ~ chi^2_n: mean n, variance 2n
    assert abs(f.mean() / sigma ** 2 - n) < 5 * math.sqrt(2 * n / lam)

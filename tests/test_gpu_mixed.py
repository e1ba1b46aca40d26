"""GPU parity of the mixed-precision path (tcgen05 TF32 / BF16 GEMMs).

The mixed path rounds the sampling operands (B D and z) to the tensor-core
input format and evaluates the objective and the rank-mu sum with 3-term split
operands; everything else is FP64. Its results are checked against the FP64
oracle with error bounds derived from the arithmetic and computed here from the
oracle's own data:
  * sample:  |dy_ik| <= (2.1 u + n 2^-24) (|B D| |Z|)_ik, u the input format's
             unit roundoff (TF32 2^-11, BF16 2^-8), FP32 accumulation;
  * objective: first-order propagation of dx plus the split-operand error
             (2^-20 TF32, 2^-14 BF16 relative to the row sums |Q| |x - x*|)
             plus the FP32 epilogue (1e-6 of the sum of |terms|);
  * update (ask/tell, same f on both sides so the ranks are identical and
    bit-exact): the sample bound carried through the weighted sums.
"""
import math

import numpy as np
import pytest

from parity_util import SEED, have_gpu, oracle_problem, oracle_state, rel, state_dict

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]

UROUND = {1: 2.0 ** -11, 2: 2.0 ** -8}        # TF32, BF16 input rounding
SPLIT = {1: 2.0 ** -20, 2: 2.0 ** -14}        # 3-term split products


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _sample_bound(d, Z, n, prec):
    BD = d["B"] * d["D"][None, :]
    u = UROUND[prec]
    return d["sigma"] * (2.1 * u + n * 2.0 ** -24) * (np.abs(BD) @ np.abs(Z))


def _grad_terms(kind, p, X):
    """|df/du_i| per row and candidate, and the largest curvature."""
    U = p.Q @ (X - p.xstar[:, None])
    if kind == 1:
        G = 2.0 * p.lamdiag[:, None] * U
        L = 2.0 * p.lamdiag.max()
    else:
        G = 2.0 * U + 20.0 * np.pi * np.sin(2.0 * np.pi * U)
        L = 2.0 + 40.0 * np.pi ** 2
    return G, L


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n,lam,kind", [(10, 10, 1), (100, 544, 2), (65, 130, 1), (130, 300, 2),
                                         (160, 320, 1), (300, 300, 2)])
def test_mixed_builtin_generation_sample_and_objective(prec, n, lam, kind):
    import paper_2409_11765_gb300 as eng
    from oracle import cmaes, objectives, philox
    from paper_2409_11765_gb300 import workloads as W
    p = W.make_problem(kind, n, SEED, 800 + n)
    d = W.random_state(n, SEED, 800 + n, cond=1e3)
    opt = eng.cmaes_default_options(precision=prec, eig_every=1, max_restarts=0)
    h = eng.cmaes_create(n, lam, d["m"], 1.0, SEED, opt)
    try:
        eng.cmaes_set_problem(h, 0, p.kind, p.Q, p.lamdiag, p.xstar)
        eng.cmaes_set_state(h, 0, state_dict(d, n, lam, gen=3))
        eng.cmaes_step_batch(h, 1)
        eng.cmaes_sync(h)
        X, f, order = eng.cmaes_get_generation(h, 0, n)
        g = eng.cmaes_get_state(h, 0, n)
    finally:
        eng.cmaes_destroy(h)
    st = oracle_state(d, n, lam, 1.0, gen=3)
    Z = philox.normals(SEED, 0, 0, 3, n, lam)
    Y, Xo = cmaes.sample(st, Z)
    bound = _sample_bound(d, Z, n, prec) + 1e-14 * np.abs(Xo)
    dx = np.abs(X - Xo)
    assert np.all(dx <= bound), ("x", float((dx / bound).max()))
    fo = oracle_problem(p)(Xo)
    G, L = _grad_terms(kind, p, Xo)
    dxn = np.linalg.norm(bound, axis=0)
    grad = np.linalg.norm(p.Q.T @ G, axis=0)
    rowsum = np.abs(p.Q) @ np.abs(Xo - p.xstar[:, None])
    split = 2.0 * SPLIT[prec] * np.sum(np.abs(G) * rowsum, axis=0)
    # FP32 epilogue (Kahan sum of the terms): a few FP32 ulps of their sum
    mag = objectives.magnitude(kind, Xo, p.Q, p.lamdiag, p.xstar)
    fbound = 1.5 * (grad * dxn + 0.5 * L * dxn ** 2) + split + 1e-6 * mag + 1e-12 * np.abs(fo)
    df = np.abs(f - fo)
    assert np.all(df <= fbound), ("f", float((df / fbound).max()))
    # the order is a valid ranking of the GPU's own values
    assert sorted(order) == list(range(lam))
    assert np.all(np.diff(f[order]) >= 0)
    # state stays valid; the best point carries its FP64 value
    assert g["gen"] == 4 and np.array_equal(g["C"], g["C"].T)
    assert np.abs(g["B"].T @ g["B"] - np.eye(n)).max() <= 1e-13 * max(n, 10)
    # the eigendecomposition (FP32 sweeps + FP64 finish on this route) is an
    # FP64-accurate decomposition of the C it was given
    recon = (g["B"] * g["D"] ** 2) @ g["B"].T
    assert rel(recon, g["C"]) <= 1e-12, rel(recon, g["C"])
    assert np.all(np.diff(g["D"]) >= 0)
    i0 = order[0]
    f_exact = oracle_problem(p)(X[:, i0:i0 + 1])[0]
    assert math.isclose(g["best_f"], f_exact, rel_tol=1e-12, abs_tol=1e-12 * abs(fo).max())


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n,lam", [(10, 12), (100, 1088)])
def test_mixed_ask_tell_update(prec, n, lam):
    """Same f on both sides: identical ranks (bit-exact), and the update
    quantities within the sample bound carried through the weighted sums."""
    import paper_2409_11765_gb300 as eng
    from oracle import cmaes, philox
    from oracle.params import Params
    from paper_2409_11765_gb300 import workloads as W
    p = W.make_problem(1, n, SEED, 900 + n, cond=1e3)
    d = W.random_state(n, SEED, 900 + n, cond=1e3)
    opt = eng.cmaes_default_options(precision=prec, eig_every=1, max_restarts=0)
    st = oracle_state(d, n, lam, 1.0, gen=2)
    Z = philox.normals(SEED, 0, 0, 2, n, lam)
    Y, Xo = cmaes.sample(st, Z)
    f = oracle_problem(p)(Xo)
    h = eng.cmaes_create(n, lam, d["m"], 1.0, SEED, opt)
    try:
        eng.cmaes_set_state(h, 0, state_dict(d, n, lam, gen=2))
        X = eng.cmaes_ask(h, 0, n)
        eng.cmaes_tell(h, 0, f)
        _, _, order = eng.cmaes_get_generation(h, 0, n)
        g = eng.cmaes_get_state(h, 0, n)
    finally:
        eng.cmaes_destroy(h)
    prm = Params(n, lam)
    rec = cmaes.generation(st, SEED, 0, None, cmaes.Options(eig_every=1, max_restarts=0), Z=Z, f=f)
    assert np.array_equal(order, rec["order"])
    by = _sample_bound(d, Z, n, prec) / d["sigma"]          # bound on |dy|
    sel = rec["order"][:prm.mu]
    w = prm.weights
    dyw = by[:, sel] @ w                                     # bound on |d<y>_w|
    u = UROUND[prec]
    dzw = u * (np.abs(Z[:, sel]) @ w)                        # bound on |d<z>_w|
    tol = 1e-13
    assert np.all(np.abs(g["m"] - st.m) <= d["sigma"] * dyw + tol * np.abs(st.m) + 1e-15)
    coef_s = math.sqrt(prm.cs * (2 - prm.cs) * prm.mueff)
    dps = coef_s * (np.abs(d["B"]) @ dzw)
    assert np.all(np.abs(g["ps"] - st.ps) <= dps + tol * np.abs(st.ps) + 1e-15)
    coef_c = math.sqrt(prm.cc * (2 - prm.cc) * prm.mueff)
    dpc = coef_c * dyw
    assert np.all(np.abs(g["pc"] - st.pc) <= dpc + tol * np.abs(st.pc) + 1e-15)
    dsig = st.sigma * (prm.cs / prm.ds) * np.linalg.norm(dps) / prm.chin * 1.01
    assert abs(g["sigma"] - st.sigma) <= dsig + 1e-13 * st.sigma
    Ys = np.abs(Y[:, sel])
    dC = prm.cmu * ((by[:, sel] * w) @ Ys.T + (Ys * w) @ by[:, sel].T
                    + 2.0 * SPLIT[prec] * (Ys * w) @ Ys.T)
    dC += prm.c1 * (np.outer(dpc, np.abs(st.pc)) + np.outer(np.abs(st.pc), dpc))
    assert np.all(np.abs(g["C"] - st.C) <= 1.01 * dC + 1e-13 * np.abs(st.C) + 1e-15)
    # eigenvalues move at most by the perturbation of C (Weyl)
    dlam = np.linalg.norm(dC, 2) * 1.01 + 1e-12 * (st.D ** 2).max()
    assert np.all(np.abs(g["D"] ** 2 - st.D ** 2) <= dlam)
    assert np.abs(g["B"].T @ g["B"] - np.eye(n)).max() <= 1e-13 * max(n, 10)
    recon = (g["B"] * g["D"] ** 2) @ g["B"].T
    assert rel(recon, g["C"]) <= 1e-12, rel(recon, g["C"])


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_small_ellipsoid_reaches_target(prec):
    """n=10, lambda=10, rotated ellipsoid cond 1e6: the mixed path reaches
    f < 1e-10 (the reported best value is an FP64 evaluation)."""
    import paper_2409_11765_gb300 as eng
    from oracle import objectives
    from paper_2409_11765_gb300 import workloads as W
    wl = W.ellipsoid_n10()
    s = wl.searches[0]
    opt = eng.cmaes_default_options(precision=prec, f_target=wl.f_target, max_restarts=0)
    h = eng.cmaes_create(s.n, s.lam, s.x0, s.sigma0, SEED, opt)
    try:
        p = s.problem
        eng.cmaes_set_problem(h, 0, p.kind, p.Q, p.lamdiag, p.xstar)
        eng.cmaes_step_batch(h, wl.generations)
        q = eng.cmaes_query(h, 0)
        x, fbest = eng.cmaes_best(h, 0, s.n)
    finally:
        eng.cmaes_destroy(h)
    f_re = objectives.evaluate(p.kind, x[:, None], p.Q, p.lamdiag, p.xstar)[0]
    assert q["done"] == 1 and (q["flags"] & 1), q
    assert fbest < 1e-10 and f_re < 1e-10
    assert math.isclose(f_re, fbest, rel_tol=1e-9, abs_tol=1e-20)


def test_mixed_kdistributed_batch_sample_bounds():
    """The benchmark's batch in TF32 mode: every level's sample within the
    bound after one generation from teacher-forced states."""
    import paper_2409_11765_gb300 as eng
    from oracle import philox
    from paper_2409_11765_gb300 import workloads as W
    n = 100
    lams = [17 << k for k in range(10)]
    p = W.make_problem(2, n, SEED, 1)
    states = [W.random_state(n, SEED, 950 + k, cond=1e2) for k in range(10)]
    opt = eng.cmaes_default_options(precision=1, eig_every=1, max_restarts=255, ipop_double=0,
                                    box_lo=-5.0, box_hi=5.0)
    h = eng.cmaes_create_batch([n] * 10, lams, [st["m"] for st in states], [2.5] * 10, SEED, opt)
    try:
        for i in range(10):
            eng.cmaes_set_problem(h, i, p.kind, p.Q, None, p.xstar)
            eng.cmaes_set_state(h, i, state_dict(states[i], n, lams[i], gen=1))
        eng.cmaes_step_batch(h, 1)
        eng.cmaes_sync(h)
        for i in (0, 4, 9):
            X, f, _ = eng.cmaes_get_generation(h, i, n)
            d = states[i]
            Z = philox.normals(SEED, i, 0, 1, n, lams[i])
            Xo = d["m"][:, None] + d["sigma"] * ((d["B"] * d["D"]) @ Z)
            bound = _sample_bound(d, Z, n, 1) + 1e-14 * np.abs(Xo)
            assert np.all(np.abs(X - Xo) <= bound), i
    finally:
        eng.cmaes_destroy(h)

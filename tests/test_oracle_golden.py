"""The oracle against the stored fixtures in tests/golden/ (each file cites
where its values come from)."""
import os

import numpy as np

from oracle import cmaes, philox
from oracle.params import Params, default_lambda

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_philox_known_answers_file():
    rows = _lines("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        vals = [int(x, 16) for x in r]
        out = philox.philox4x32_10(*vals[:4], vals[4], vals[5])
        assert [int(w) for w in out] == vals[6:]


def test_default_lambda_file():
    for n, lam in _lines("default_lambda.txt"):
        assert default_lambda(int(n)) == int(lam)


def test_n2_generation_file():
    g = {r[0]: r[1:] for r in _lines("n2_generation.txt")}
    z = np.array([[float(a) for a in p.split()] for p in " ".join(g["z"]).split(";")]).T
    f = np.array([float(x) for x in g["f"]])
    st = cmaes.State(2, 6, 1.0, np.zeros(2), 1.0)
    p = Params(2, 6)
    Y, X = cmaes.sample(st, z)
    assert np.allclose(((X - np.array([[1.0], [0.0]])) ** 2).sum(0), f, atol=0)
    rec = cmaes.update(st, p, z, Y, X, f)
    num = lambda k: np.array([float(x) for x in g[k]])
    assert list(rec["order"]) == [int(x) for x in g["order"]]
    tol = 5e-13
    assert np.allclose(p.weights, num("weights"), atol=tol)
    for k, v in (("mueff", p.mueff), ("c1", p.c1), ("cmu", p.cmu), ("cs", p.cs), ("ds", p.ds),
                 ("cc", p.cc), ("chin", p.chin), ("psnorm", rec["psnorm"]), ("hsig", rec["hsig"]),
                 ("sigma", st.sigma)):
        assert abs(v - num(k)[0]) < tol, k
    for k, v in (("m", st.m), ("ps", st.ps), ("pc", st.pc), ("C", st.C.ravel())):
        assert np.allclose(v, num(k), atol=tol), k
    assert np.allclose(np.linalg.eigvalsh(st.C), num("eig"), atol=tol)


def test_params_branches_file():
    """d_sigma on both sides of its max(0, .) branch, MaxIter and the
    TolHistFun history length against values worked out by hand."""
    rows = _lines("params_branches.txt")
    kinds = {r[0] for r in rows}
    assert kinds == {"dsigma", "maxiter", "histlen"}
    active = 0
    for r in rows:
        n, lam = int(r[1]), int(r[2])
        p = Params(n, lam)
        if r[0] == "dsigma":
            mueff, cs, inner, ds = (float(x) for x in r[3:7])
            assert abs(p.mueff - mueff) <= 5e-14 * mueff
            assert abs(p.cs - cs) <= 5e-14
            assert abs(p.ds - ds) <= 5e-14 * ds
            active += inner > 0
        elif r[0] == "maxiter":
            assert p.max_iter == int(r[3])
        else:
            assert p.hist_len == int(r[3])
    assert active == 2

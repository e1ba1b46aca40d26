"""The allocation-free objective evaluation against the oracle's objectives
and the engine's own.

cmaes_evaluate_noalloc is for callers that cannot allocate device memory at
the point they need objective values (their memory is managed by another
component, or an allocation's latency and implicit synchronisation are not
acceptable). It keeps its one intermediate in a fixed static device array.
Here it is fed the points the engine sampled in two consecutive generations
and must return, within the FP64 tolerance of the parity tests, the values the
oracle's objectives (oracle/objectives.py) give for them, and the values the
engine computed (the arithmetic is the same, so in practice bit for bit).
Padded leading dimensions (NaN in the padding) and a panel that fills the
scratch exactly are covered too. Collected last so that a run stopping at the
first failure has run everything else; it builds the library itself, so it
also passes alone.
"""
import numpy as np
import pytest

from parity_util import SEED, TOL_FP64, have_gpu, rel

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _dev(a, ld=None):
    """Column-major copy of a host matrix (or a vector) in device memory; a
    matrix gets leading dimension ld (NaN in the padding rows)."""
    import torch
    a = np.asarray(a, dtype=np.float64)
    if a.ndim == 1:
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ld = ld or a.shape[0]
    pad = np.full((a.shape[1], ld), np.nan)
    pad[:, :a.shape[0]] = a.T
    return torch.from_numpy(np.ascontiguousarray(pad)).cuda()


def _oracle_f(p, X):
    from oracle import objectives
    return objectives.evaluate(p.kind, X, p.Q, p.lamdiag, p.xstar), \
        objectives.magnitude(p.kind, X, p.Q, p.lamdiag, p.xstar)


def _eval(eng, kind, n, lam, Xd, ld, Qd, ldq, Ld, Sd):
    import torch
    fd = torch.full((lam,), float("nan"), dtype=torch.float64, device="cuda")
    eng.cmaes_evaluate_noalloc(kind, n, lam, Xd.data_ptr(), ld,
                               Qd.data_ptr() if Qd is not None else None, ldq,
                               Ld.data_ptr() if Ld is not None else None,
                               Sd.data_ptr(), fd.data_ptr(), None)
    torch.cuda.synchronize()
    return fd.cpu().numpy()


@pytest.mark.parametrize("kind,lam", [(2, 8704), (1, 544), (3, 300)])
def test_noalloc_evaluation_matches_oracle_and_engine(kind, lam):
    import paper_2409_11765_gb300 as eng
    from paper_2409_11765_gb300 import workloads as W
    n = 100
    p = W.make_problem(kind, n, SEED, 700 + kind)
    x0 = W.start_point(n, -4, 4, SEED, 700 + kind)
    h = eng.cmaes_create(n, lam, x0, 1.5, SEED, eng.cmaes_default_options(max_restarts=0))
    Qd = _dev(p.Q) if p.Q is not None else None
    Ld = _dev(p.lamdiag) if p.lamdiag is not None else None
    Sd = _dev(p.xstar)
    try:
        eng.cmaes_set_problem(h, 0, p.kind, p.Q, p.lamdiag, p.xstar)
        for call in range(2):                 # two calls in a row, new points each time
            eng.cmaes_step_batch(h, 1)
            X, f_engine, _ = eng.cmaes_get_generation(h, 0, n)
            f = _eval(eng, kind, n, lam, _dev(X), n, Qd, n, Ld, Sd)
            assert np.all(np.isfinite(f)), call
            fo, mag = _oracle_f(p, X)
            assert (np.abs(f - fo) / mag).max() <= TOL_FP64, call
            assert rel(f, f_engine) <= TOL_FP64, (call, rel(f, f_engine))
    finally:
        eng.cmaes_destroy(h)


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_noalloc_padded_leading_dimensions(kind):
    """ld = n + 3 for X and ldq = n + 5 for Q, NaN in every padding row: the
    padding is never read, and f equals the oracle's."""
    import paper_2409_11765_gb300 as eng
    from paper_2409_11765_gb300 import workloads as W
    n, lam = 77, 130
    p = W.make_problem(kind, n, SEED, 720 + kind)
    X = W.rng_for(SEED, 721, kind).uniform(-4, 4, size=(n, lam))
    Qd = _dev(p.Q, n + 5) if p.Q is not None else None
    Ld = _dev(p.lamdiag) if p.lamdiag is not None else None
    f = _eval(eng, kind, n, lam, _dev(X, n + 3), n + 3, Qd, n + 5, Ld, _dev(p.xstar))
    fo, mag = _oracle_f(p, X)
    assert np.all(np.isfinite(f))
    assert (np.abs(f - fo) / mag).max() <= TOL_FP64


def test_noalloc_panel_that_fills_the_scratch_exactly():
    """ld * lambda == 2^20 doubles: the largest accepted rotated panel."""
    import paper_2409_11765_gb300 as eng
    from paper_2409_11765_gb300 import workloads as W
    n, ld, lam = 120, 128, 8192                  # 128 * 8192 = 2^20
    p = W.make_problem(2, n, SEED, 730)
    X = W.rng_for(SEED, 731).uniform(-4, 4, size=(n, lam))
    f = _eval(eng, 2, n, lam, _dev(X, ld), ld, _dev(p.Q), n, None, _dev(p.xstar))
    fo, mag = _oracle_f(p, X)
    assert (np.abs(f - fo) / mag).max() <= TOL_FP64


def test_noalloc_rejects_oversize_panel():
    import torch
    import paper_2409_11765_gb300 as eng
    n, lam = 128, 8193                        # 128 * 8193 > 2^20 doubles of scratch
    X = torch.zeros(n * lam, dtype=torch.float64, device="cuda")
    Q = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    s = torch.zeros(n, dtype=torch.float64, device="cuda")
    f = torch.zeros(lam, dtype=torch.float64, device="cuda")
    with pytest.raises(eng.CmaesError) as e:
        eng.cmaes_evaluate_noalloc(2, n, lam, X.data_ptr(), n, Q.data_ptr(), n, None,
                                   s.data_ptr(), f.data_ptr(), None)
    assert e.value.status == 1 and "exceeds" in str(e.value)

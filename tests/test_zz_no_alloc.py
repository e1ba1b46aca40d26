"""The allocation-free objective evaluation against the engine's own.

cmaes_evaluate_noalloc is for callers that cannot allocate device memory at
the point they need objective values (their memory is managed by another
component, or an allocation's latency and implicit synchronisation are not
acceptable). It keeps its one intermediate in a fixed static device array.
Here it is fed the points the engine sampled in two consecutive generations
and must return the values the engine computed for them, within the FP64
tolerance of the parity tests (the arithmetic is the same, so in practice bit
for bit). Collected last so that a run stopping at the first failure has run
everything else; it builds the library itself, so it also passes alone.
"""
import numpy as np
import pytest

from parity_util import SEED, TOL_FP64, have_gpu, rel

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not have_gpu(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _dev(a):
    """Column-major copy of a host matrix (or a vector) in device memory."""
    import torch
    a = np.asarray(a, dtype=np.float64)
    host = np.ascontiguousarray(a.T) if a.ndim == 2 else np.ascontiguousarray(a)
    return torch.from_numpy(host).cuda()


@pytest.mark.parametrize("kind,lam", [(2, 8704), (1, 544), (3, 300)])
def test_noalloc_evaluation_matches_engine(kind, lam):
    import torch
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
            Xd = _dev(X)
            fd = torch.full((lam,), float("nan"), dtype=torch.float64, device="cuda")
            eng.cmaes_evaluate_noalloc(kind, n, lam, Xd.data_ptr(), n,
                                       Qd.data_ptr() if Qd is not None else None, n,
                                       Ld.data_ptr() if Ld is not None else None,
                                       Sd.data_ptr(), fd.data_ptr(), None)
            torch.cuda.synchronize()
            f = fd.cpu().numpy()
            assert np.all(np.isfinite(f)), call
            assert rel(f, f_engine) <= TOL_FP64, (call, rel(f, f_engine))
    finally:
        eng.cmaes_destroy(h)


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

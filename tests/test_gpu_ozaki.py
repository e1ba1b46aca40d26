"""The FP64-accurate tensor-core product (include/cmaes_ozaki.h) against exact
and extended-precision references on seeded inputs: integer matrices whose
product is exact in FP64 must come out bit-exact; general FP64 matrices (rows
and columns of very different scales, ragged sizes, K across several exact
chunks) must agree with a long-double product to within the representation
bound the header states."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def eng():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2409_11765_gb300 as e
    return e


def _dev(a):
    return torch.from_numpy(np.asfortranarray(a)).cuda()


def _run(eng, A, B, C=None, alpha=1.0, beta=0.0):
    M, K = A.shape
    N = B.shape[1]
    dA, dB = _dev(A), _dev(B)
    dC = _dev(C if C is not None else np.zeros((M, N)))
    eng.cmaes_ozaki_dgemm(M, N, K, alpha, dA.data_ptr(), M, dB.data_ptr(), K, beta, dC.data_ptr(), M)
    torch.cuda.synchronize()
    return np.asfortranarray(dC.cpu().numpy())


def _bound(A, B):
    # the header's bound: representation 2^(a-55) per entry of A (2^a the
    # row's power-of-two bound) and 2^(b-55) per entry of B, dropped digit
    # products 6 * 2^(a+b-54) per K term, the light buckets, FP64 rounding
    ra = 2.0 ** np.ceil(np.log2(np.max(np.abs(A), axis=1, keepdims=True) * (1 + 2.0 ** -52) + 1e-300))
    cb = 2.0 ** np.ceil(np.log2(np.max(np.abs(B), axis=0, keepdims=True) * (1 + 2.0 ** -52) + 1e-300))
    K = A.shape[1]
    rep = 2.0 ** -55 * (ra * np.sum(np.abs(B), axis=0, keepdims=True)
                        + np.sum(np.abs(A), axis=1, keepdims=True) * cb)
    dropped = (6 * 2.0 ** -54 + 2.0 ** -48) * K * ra * cb
    return rep + dropped + 2 * 2.0 ** -53 * (np.abs(A) @ np.abs(B))


@pytest.mark.parametrize("M,N,K", [(200, 150, 300), (130, 1, 5), (1, 70, 1000), (257, 129, 640)])
def test_integer_products_are_exact(eng, M, N, K):
    rng = np.random.default_rng(11 + M + N + K)
    A = rng.integers(-2048, 2049, size=(M, K)).astype(np.float64)
    B = rng.integers(-2048, 2049, size=(K, N)).astype(np.float64)
    C = _run(eng, A, B)
    exact = A.astype(np.int64) @ B.astype(np.int64)
    assert np.array_equal(C, exact.astype(np.float64))


@pytest.mark.parametrize("M,N,K", [(300, 257, 1000), (64, 64, 33), (129, 200, 2048), (128, 64, 4096)])
def test_scaled_products_within_bound(eng, M, N, K):
    rng = np.random.default_rng(5 * M + N + K)
    A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-6, 6, size=(M, 1))
    B = rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-6, 6, size=(1, N))
    A[:, ::7] *= 1e-9  # entries far below their row's largest
    C = _run(eng, A, B)
    ref = (A.astype(np.longdouble) @ B.astype(np.longdouble)).astype(np.float64)
    err = np.abs(C - ref)
    assert np.all(err <= _bound(A, B)), float(np.max(err / _bound(A, B)))


def test_orthogonal_gram_to_fp64_rounding(eng):
    rng = np.random.default_rng(3)
    n = 700
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    G = _run(eng, Q.T.copy(), Q, C=np.eye(n), alpha=1.0, beta=-1.0)  # Q^T Q - I
    ref = (Q.T.astype(np.longdouble) @ Q.astype(np.longdouble) - np.eye(n)).astype(np.float64)
    assert np.max(np.abs(G - ref)) <= 64 * 2.0 ** -53
    assert np.max(np.abs(G)) <= 1e-13


def test_alpha_beta_zero_rows_and_wide_range(eng):
    rng = np.random.default_rng(8)
    M, N, K = 150, 90, 400
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    A[3] = 0.0
    B[:, 5] = 0.0
    A[7] *= 1e200
    A[8] *= 1e-200
    C0 = rng.standard_normal((M, N))
    C = _run(eng, A, B, C=C0, alpha=2.0, beta=-0.5)
    ref = (2.0 * (A.astype(np.longdouble) @ B.astype(np.longdouble)) - 0.5 * C0).astype(np.float64)
    assert np.all(C[3] == -0.5 * C0[3])
    assert np.all(C[:, 5] == -0.5 * C0[:, 5])
    bound = 2.0 * _bound(A, B) + 2.0 ** -52 * np.abs(ref)
    assert np.all(np.abs(C - ref) <= bound)

"""Index algebra of the ring-moved FP32 Jacobi layout (CPU, no GPU).

The FP32 Jacobi kernels move the matrix with the round-robin ring instead of
addressing it through the ring. These tests pin the facts they rely on,
each restated here from its definition:
- the round-robin (circle-method) pairing and the one-place ring turn;
- the block of step r that holds each pair's pivot at step r + 1 (role blocks);
- the thread lists (role blocks first) cover every off-diagonal block once;
- the packed diagonal-major slot order and its inverse;
- a plain Jacobi on the moved layout gives the same rotations as on the
  fixed one (small sizes, FP64, pure Python).
"""
import math

import numpy as np
import pytest


def rr_pair(r, k, M):
    """Pair k of round-robin step r over N = M + 1 players (player M fixed)."""
    return (r, M) if k == 0 else ((r + k) % M, (r - k) % M)


def ring_next(K, x, P):
    """Ring position (pair, role a = 0 / b = 1) at step r + 1 of position (K, x) at step r."""
    if x == 0:
        return (K - 1, 0) if K >= 1 else (1, 1)
    if K == 0:
        return (0, 1)
    if K == P - 1:
        return (P - 1, 0)
    return (K + 1, 1)


def role(Pi, Qi, P):
    """(next pair, entry) whose pivot block (Pi, Qi) holds; entry 0/2/3 = (a,a)/(b,a)/(b,b)."""
    if (Pi, Qi) == (0, 1):
        return 0, 2
    if (Pi, Qi) == (0, 2):
        return 1, 0
    if Qi == Pi + 2:
        return Pi + 1, 2
    if (Pi, Qi) == (P - 2, P - 1):
        return P - 1, 3
    return None


def role_block(k, P):
    return (0, 1) if k == 0 else (0, 2) if k == 1 else (P - 2, P - 1) if k == P - 1 else (k - 1, k + 1)


def dbase(d, P):
    return (d - 3) * P - ((d - 1) * d // 2 - 3)


def slot(K, L, P):
    """Packed diagonal-major slot of off-diagonal block (K, L), K < L."""
    d = L - K
    if d == 2:
        return K + 1
    if d == 1:
        return 0 if K == 0 else (P - 1 if K == P - 2 else P + K - 1)
    return P + (P - 3) + dbase(d, P) + K


def block(k, P):
    """Inverse of slot(): the quadratic root for the diagonal, then at most two fix-ups."""
    if k < P:
        return role_block(k, P)
    j = k - P
    if j < P - 3:
        return (j + 1, j + 2)
    j -= P - 3
    b = 2.0 * P + 1.0
    d = max(3, int((b - math.sqrt(max(b * b - 4.0 * (6.0 * P - 6.0 + 2.0 * j), 0.0))) * 0.5))
    while d + 1 <= P - 1 and dbase(d + 1, P) <= j:
        d += 1
    while d > 3 and dbase(d, P) > j:
        d -= 1
    K = j - dbase(d, P)
    return (K, K + d)


@pytest.mark.parametrize("N", [4, 6, 34, 100, 160, 322])
def test_ring_turn_matches_round_robin(N):
    M, P = N - 1, N // 2
    for r in range(M):
        r1 = (r + 1) % M
        for k in range(P):
            for x in (0, 1):
                e = rr_pair(r, k, M)[x]
                K1, x1 = ring_next(k, x, P)
                assert rr_pair(r1, K1, M)[x1] == e
        # every player plays exactly once per step
        assert sorted(v for k in range(P) for v in rr_pair(r, k, M)) == list(range(N))


@pytest.mark.parametrize("N", [8, 10, 34, 100, 170])
def test_role_blocks_hold_the_next_pivots(N):
    M, P = N - 1, N // 2
    for r in range(M):
        seen = {}
        for Qi in range(P):
            for Pi in range(Qi):
                ro = role(Pi, Qi, P)
                if ro is None:
                    continue
                k, ent = ro
                assert (Pi, Qi) == role_block(k, P)
                x, y = ent >> 1, ent & 1
                (K1, x1), (L1, y1) = ring_next(Pi, x, P), ring_next(Qi, y, P)
                assert K1 == L1 == k and {x1, y1} == {0, 1}  # lands on pair k's off-diagonal entry
                seen[k] = (Pi, Qi)
        assert sorted(seen) == list(range(P))


@pytest.mark.parametrize("P", [17, 50, 80])
def test_thread_lists_cover_every_block_once(P):
    NT = 1024
    nblk = P * (P - 1) // 2
    kmax = 1 + (nblk - NT + (NT - P) - 1) // (NT - P) if nblk > NT else 1
    ks = []
    for tid in range(NT):
        for u in range(max(kmax, 1)):
            k = tid if u == 0 else (NT + (NT - P) * (u - 1) + tid - P if tid >= P else nblk)
            if k < nblk:
                ks.append(k)
    assert sorted(ks) == list(range(nblk))
    assert all(ks.count(k) == 1 for k in range(P))  # the role threads own one block each


@pytest.mark.parametrize("P", [4, 5, 17, 81, 100, 300])
def test_packed_slots_are_a_bijection(P):
    nb = P * (P - 1) // 2
    got = [block(k, P) for k in range(nb)]
    assert sorted(got) == sorted((i, j) for j in range(P) for i in range(j))
    for k, (K, L) in enumerate(got):
        assert slot(K, L, P) == k
    assert all(role(*got[k], P) is not None for k in range(P))  # role blocks first


def _jacobi_rotation(app, aqq, apq):
    theta = (aqq - app) / (2.0 * apq)
    t = (1.0 if theta >= 0 else -1.0) / (abs(theta) + math.sqrt(theta * theta + 1.0))
    c = 1.0 / math.sqrt(t * t + 1.0)
    return c, t * c, t


@pytest.mark.parametrize("n", [6, 7, 12])
def test_moved_layout_gives_the_same_rotations(n):
    """Two sweeps of cyclic Jacobi, once on A indexed through the ring and
    once on the entries moved with the ring: identical rotation tables."""
    rng = np.random.default_rng(n)
    G = rng.standard_normal((n, n))
    A0 = (G + G.T) / 2.0
    N = n + (n & 1)
    P, M = N // 2, N - 1
    Af = np.zeros((N, N))
    Af[:n, :n] = A0
    steps = 2 * M

    def rotates(app, aqq, apq):
        return abs(apq) > 1e-12 and apq * apq > 1e-20 * abs(app * aqq)

    # fixed storage, moving indices
    A = Af.copy()
    log1 = []
    for t in range(steps):
        r = t % M
        rec = []
        for k in range(P):
            p, q = rr_pair(r, k, M)
            c, s = 1.0, 0.0
            if p < n and q < n and rotates(A[p, p], A[q, q], A[p, q]):
                c, s, _ = _jacobi_rotation(A[p, p], A[q, q], A[p, q])
            rec.append((c, s))
        J = np.eye(N)
        for k, (c, s) in enumerate(rec):
            p, q = rr_pair(r, k, M)
            J[p, p], J[q, q], J[p, q], J[q, p] = c, c, s, -s
        A = J.T @ A @ J
        log1.append(rec)

    # moved storage: entry between positions (K, x), (L, y) at [2K + x, 2L + y]
    pos = np.zeros((N, N))
    where = {}
    for k in range(P):
        p, q = rr_pair(0, k, M)
        where[(k, 0)], where[(k, 1)] = p, q
    for (K, x), e in where.items():
        for (L, y), f in where.items():
            pos[2 * K + x, 2 * L + y] = Af[e, f]
    log2 = []
    for t in range(steps):
        r = t % M
        rec = []
        for k in range(P):
            p, q = rr_pair(r, k, M)
            app, aqq, apq = pos[2 * k, 2 * k], pos[2 * k + 1, 2 * k + 1], pos[2 * k, 2 * k + 1]
            c, s = 1.0, 0.0
            if p < n and q < n and rotates(app, aqq, apq):
                c, s, _ = _jacobi_rotation(app, aqq, apq)
            rec.append((c, s))
        J = np.eye(N)
        for k, (c, s) in enumerate(rec):
            J[2 * k, 2 * k], J[2 * k + 1, 2 * k + 1], J[2 * k, 2 * k + 1], J[2 * k + 1, 2 * k] = c, c, s, -s
        rot = J.T @ pos @ J
        nxt = np.zeros_like(rot)
        for K in range(P):
            for x in (0, 1):
                K1, x1 = ring_next(K, x, P)
                for L in range(P):
                    for y in (0, 1):
                        L1, y1 = ring_next(L, y, P)
                        nxt[2 * K1 + x1, 2 * L1 + y1] = rot[2 * K + x, 2 * L + y]
        pos = nxt
        log2.append(rec)
    np.testing.assert_allclose(np.array(log1), np.array(log2), rtol=0, atol=1e-12)

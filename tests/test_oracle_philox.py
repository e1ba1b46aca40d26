"""Pins for the oracle's counter-based generator and normal transform."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import philox


# Known-answer values published with the Random123 library (kat_vectors,
# philox4x32 with 10 rounds) for the generator of Salmon et al., SC'11.
KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


@pytest.mark.parametrize("ctr,key,expect", KAT)
def test_philox_known_answers(ctr, key, expect):
    out = philox.philox4x32_10(*ctr, *key)
    assert tuple(int(w) for w in out) == expect


def test_philox_vectorised_matches_scalar():
    c0 = np.arange(5, dtype=np.uint64)
    vec = philox.philox4x32_10(c0, 7, 11, 13, 0x1234, 0x5678)
    for j in range(5):
        sc = philox.philox4x32_10(j, 7, 11, 13, 0x1234, 0x5678)
        assert all(int(v[j]) == int(s) for v, s in zip(vec, sc))


def test_uniform_open_interval_and_exact():
    wa = np.array([0, 0xffffffff, 0x80000000, 0], dtype=np.uint64)
    wb = np.array([0, 0xffffffff, 0, 0xfff], dtype=np.uint64)
    u = philox.uniform_from_words(wa, wb)
    assert np.all(u > 0.0) and np.all(u < 1.0)
    # u * 2^52 - 1/2 is the integer made of the top 52 bits
    v = u * 2.0 ** 52 - 0.5
    assert np.all(v == np.floor(v))
    assert u[0] == 0.5 * 2.0 ** -52
    assert u[2] == 0.5 + 0.5 * 2.0 ** -52
    # the low 12 bits of the second word are dropped
    assert u[3] == u[0]


def test_box_muller_invariants():
    seed, s, r, g, n, lam = 99, 3, 1, 5, 6, 40
    Z = philox.normals(seed, s, r, g, n, lam)
    k0, k1 = philox.seed_key(seed)
    for k in (0, 17, 39):
        for j in range(n // 2):
            w = philox.philox4x32_10(j, k, g, philox.stream_word(s, r), k0, k1)
            u1 = float(philox.uniform_from_words(w[0], w[1]))
            u2 = float(philox.uniform_from_words(w[2], w[3]))
            z0, z1 = Z[2 * j, k], Z[2 * j + 1, k]
            assert math.isclose(z0 * z0 + z1 * z1, -2.0 * math.log(u1), rel_tol=1e-14)
            ang = math.atan2(z1, z0) % (2 * math.pi)
            assert math.isclose(ang, (2 * math.pi * u2) % (2 * math.pi), rel_tol=0, abs_tol=1e-12)


def test_normals_distribution():
    Z = philox.normals(20240918, 0, 0, 0, 500, 2000).ravel()
    N = Z.size
    assert abs(Z.mean()) < 5.0 / math.sqrt(N)
    assert abs(Z.var() - 1.0) < 5.0 * math.sqrt(2.0 / N)
    assert stats.kstest(Z, "norm").pvalue > 1e-4
    # cosine and sine branches are each standard normal and uncorrelated
    Zm = philox.normals(7, 1, 0, 3, 2, 200000)
    assert abs(np.corrcoef(Zm[0], Zm[1])[0, 1]) < 5.0 / math.sqrt(200000)


def test_streams_are_distinct_and_reproducible():
    a = philox.normals(1, 0, 0, 0, 8, 8)
    assert np.array_equal(a, philox.normals(1, 0, 0, 0, 8, 8))
    for other in (philox.normals(2, 0, 0, 0, 8, 8), philox.normals(1, 1, 0, 0, 8, 8),
                  philox.normals(1, 0, 1, 0, 8, 8), philox.normals(1, 0, 0, 1, 8, 8)):
        assert not np.any(a == other)
    # a larger population extends the smaller one column by column
    assert np.array_equal(philox.normals(1, 0, 0, 0, 8, 20)[:, :8], a)
    # odd n uses the first n coordinates of the even-n draw
    assert np.array_equal(philox.normals(1, 0, 0, 0, 7, 8), a[:7])


def test_restart_mean_in_box_and_uniform():
    m = philox.restart_mean(5, 2, 3, 20000, -5.0, 5.0)
    assert np.all(m > -5.0) and np.all(m < 5.0)
    assert stats.kstest((m + 5.0) / 10.0, "uniform").pvalue > 1e-4
    assert not np.array_equal(m, philox.restart_mean(5, 2, 4, 20000, -5.0, 5.0))


def test_normals_columns_match_full_draw():
    full = philox.normals(3, 2, 1, 7, 9, 40)
    cols = [0, 5, 39, 17]
    assert np.array_equal(philox.normals_columns(3, 2, 1, 7, 9, cols), full[:, cols])

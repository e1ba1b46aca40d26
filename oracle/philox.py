"""Philox4x32-10 and the Box-Muller normal transform (oracle side).

Test infrastructure: see the package docstring.

The paper draws the points of Eq. (1) from N(0, I) but leaves the generator to
the c-cmaes code and seeds each descent with "time x MPI rank" (§3.2.2). Here
every random number is a pure function of a counter, so any candidate's z can
be regenerated anywhere: the generator is Philox4x32 with 10 rounds, written
from its published definition (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11, §3.3 / Fig. 2):

  round:  (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2   (32x32 -> 64 bit)
          c' = (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)
  key schedule between rounds: k0 += 0x9E3779B9, k1 += 0xBB67AE85
  multipliers M0 = 0xD2511F53, M1 = 0xCD9E8D57.

Counter layout used by both the oracle and the engine (a reading of ours; the
paper fixes none):

  z_{k,i} of search s, descent r, generation g:
      counter = (i >> 1, k, g, (s << 8) | (r & 255)),  key = (seed_lo, seed_hi)
      words (w0, w1) -> u1, (w2, w3) -> u2; i even takes the cosine branch,
      i odd the sine branch of Box-Muller.
  initial mean of descent r >= 1 (Algorithm 2, "initialize"):
      counter = (i >> 1, 0xFFFFFFFF, 0xFFFFFFFF, (s << 8) | (r & 255)),
      i even takes u(w0, w1), i odd u(w2, w3);  m_i = lo + (hi - lo) * u.

Uniform from two words: v = ((wa << 32) | wb) >> 12 (52 bits),
u = (v + 0.5) * 2^-52, which lies in (0, 1) and is exact in FP64.
Normal pair: r = sqrt(-2 ln u1), a = (2 pi) * u2, z = (r cos a, r sin a).
"""
import numpy as np

MASK32 = 0xFFFFFFFF
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MEAN_STREAM = 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four output words for counters (c0..c3) under key (k0, k1).

    Counters may be numpy arrays (broadcast together); keys are scalars.
    Products of two 32-bit values fit in uint64 exactly, so the high and low
    halves are taken by shifting and masking.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & np.uint64(MASK32)
                      for c in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = int(k0) & MASK32
    k1 = int(k1) & MASK32
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    s32 = np.uint64(32)
    mask = np.uint64(MASK32)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = m0 * c0
        p1 = m1 * c2
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
    return c0, c1, c2, c3


def seed_key(seed):
    """Split a 64-bit seed into the two 32-bit Philox key words."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & MASK32, (seed >> 32) & MASK32


def uniform_from_words(wa, wb):
    """52-bit uniform in the open interval (0, 1) from two 32-bit words."""
    v = ((np.asarray(wa, dtype=np.uint64) << np.uint64(32))
         | np.asarray(wb, dtype=np.uint64)) >> np.uint64(12)
    return (v.astype(np.float64) + 0.5) * 2.0 ** -52


def stream_word(search, restart):
    """Fourth counter word: search index and descent number."""
    return ((int(search) << 8) | (int(restart) & 255)) & MASK32


def normals(seed, search, restart, gen, n, lam):
    """Z (n x lam, FP64) of one generation: the z_k of Eq. (1), column k."""
    k0, k1 = seed_key(seed)
    i = np.arange(n, dtype=np.uint64)[:, None]
    k = np.arange(lam, dtype=np.uint64)[None, :]
    w0, w1, w2, w3 = philox4x32_10(i >> np.uint64(1), k, gen,
                                   stream_word(search, restart), k0, k1)
    u1 = uniform_from_words(w0, w1)
    u2 = uniform_from_words(w2, w3)
    r = np.sqrt(-2.0 * np.log(u1))
    a = (2.0 * np.pi) * u2
    even = (np.arange(n) % 2 == 0)[:, None]
    return np.where(even, r * np.cos(a), r * np.sin(a))


def normals_columns(seed, search, restart, gen, n, cols):
    """Columns `cols` of normals(seed, search, restart, gen, n, lam): the same
    counters, for when only a few candidates are needed."""
    k0, k1 = seed_key(seed)
    i = np.arange(n, dtype=np.uint64)[:, None]
    k = np.asarray(cols, dtype=np.uint64)[None, :]
    w0, w1, w2, w3 = philox4x32_10(i >> np.uint64(1), k, gen,
                                   stream_word(search, restart), k0, k1)
    u1 = uniform_from_words(w0, w1)
    u2 = uniform_from_words(w2, w3)
    r = np.sqrt(-2.0 * np.log(u1))
    a = (2.0 * np.pi) * u2
    even = (np.arange(n) % 2 == 0)[:, None]
    return np.where(even, r * np.cos(a), r * np.sin(a))


def restart_mean(seed, search, restart, n, lo, hi):
    """Initial mean of descent `restart`: uniform in the box [lo, hi]^n."""
    k0, k1 = seed_key(seed)
    i = np.arange(n, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32_10(i >> np.uint64(1), MEAN_STREAM, MEAN_STREAM,
                                   stream_word(search, restart), k0, k1)
    u_even = uniform_from_words(w0, w1)
    u_odd = uniform_from_words(w2, w3)
    u = np.where(np.arange(n) % 2 == 0, u_even, u_odd)
    return lo + (hi - lo) * u

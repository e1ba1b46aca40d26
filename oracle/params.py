"""Strategy parameters of CMA-ES as functions of (n, lambda) (oracle side).

Test infrastructure: see the package docstring.

The paper keeps the c-cmaes defaults for every parameter except the initial
mean, the initial step size and lambda_start (§4.1), and it requires only that
the rank weights w_rk(i) favour better points and sum to one (§2.1, Eq. (2)).
Our reading takes the published defaults of Hansen's CMA-ES tutorial
(arXiv:1604.00772) with positive weights on the best mu = floor(lambda/2)
points and zero weight on the rest, which makes Eq. (2)'s sum over all lambda
points a sum over the mu selected ones.
"""
import math

import numpy as np


def default_lambda(n):
    """Default population size 4 + floor(3 ln n) (tutorial default)."""
    return 4 + int(math.floor(3.0 * math.log(n)))


def expected_norm(n):
    """E||N(0, I_n)|| ~ sqrt(n) (1 - 1/(4n) + 1/(21 n^2))."""
    return math.sqrt(n) * (1.0 - 1.0 / (4.0 * n) + 1.0 / (21.0 * n * n))


class Params:
    """All strategy constants of one descent with dimension n and size lam."""

    def __init__(self, n, lam):
        if n < 1 or lam < 2:
            raise ValueError("need n >= 1 and lambda >= 2")
        self.n = n
        self.lam = lam
        self.mu = lam // 2
        i = np.arange(1, self.mu + 1, dtype=np.float64)
        wprime = math.log((lam + 1) / 2.0) - np.log(i)
        # Eq. (2): weights decrease with rank and sum to one.
        self.weights = wprime / wprime.sum()
        self.mueff = 1.0 / float(np.sum(self.weights ** 2))
        mueff = self.mueff
        self.cs = (mueff + 2.0) / (n + mueff + 5.0)
        self.ds = (1.0 + 2.0 * max(0.0, math.sqrt((mueff - 1.0) / (n + 1.0)) - 1.0)
                   + self.cs)
        self.cc = (4.0 + mueff / n) / (n + 4.0 + 2.0 * mueff / n)
        self.c1 = 2.0 / ((n + 1.3) ** 2 + mueff)
        self.cmu = min(1.0 - self.c1,
                       2.0 * (mueff - 2.0 + 1.0 / mueff) / ((n + 2.0) ** 2 + mueff))
        self.chin = expected_norm(n)
        # Lazy eigendecomposition cadence (the O(n^3) step of §2.1 is amortised
        # over 1 / ((c1 + cmu) n 10) generations, at least one).
        self.g_eig = max(1, int(math.floor(1.0 / ((self.c1 + self.cmu) * n * 10.0))))
        # Length of the best-f history behind the "quality not improving" stop.
        self.hist_len = 10 + int(math.ceil(30.0 * n / lam))
        # Default per-descent iteration cap ("MaxIter").
        self.max_iter = int(math.floor(100.0 + 50.0 * (n + 3.0) ** 2 / math.sqrt(lam)))

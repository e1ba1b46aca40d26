"""Seeded synthetic problem instances and search configurations.

This module only draws inputs: objective instances (Haar-orthogonal rotation
Q, diagonal Lambda, optimum x*) and starting points. It holds none of the
CMA-ES arithmetic, so both the CUDA engine's tests and the CPU oracle can take
their inputs from it.

The paper benchmarks on the BBOB suite (§4.1), which is not available here; the
stand-ins are seeded instances of the same families: a rotated ill-conditioned
ellipsoid (BBOB's f10 family), a rotated Rastrigin (f15 family) and a
separable sphere (f1). Initial means are uniform in the search box and the
initial step size is a quarter of the box width, as in §4.1.
"""
import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED = 20240918

ELLIPSOID = 1
RASTRIGIN = 2
SPHERE = 3


def rng_for(seed, *stream):
    """Independent numpy generator for (seed, stream ids)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, *stream])))


def haar_orthogonal(n, rng):
    """Haar-distributed orthogonal matrix: QR of a Gaussian matrix with the
    signs of R's diagonal moved into Q (Mezzadri 2007)."""
    A = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(R))[None, :]
    return np.ascontiguousarray(Q)


def ellipsoid_diag(n, cond):
    """Lambda_ii = cond^((i-1)/(n-1)), i = 1..n."""
    if n == 1:
        return np.ones(1)
    return cond ** (np.arange(n, dtype=np.float64) / (n - 1))


def default_lambda(n):
    """4 + floor(3 ln n), used to size configurations."""
    return 4 + int(math.floor(3.0 * math.log(n)))


@dataclass
class ProblemInstance:
    kind: int
    n: int
    xstar: np.ndarray
    Q: Optional[np.ndarray] = None
    lamdiag: Optional[np.ndarray] = None


def make_problem(kind, n, seed=SEED, stream=0, cond=1e6, lo=-4.0, hi=4.0):
    rng = rng_for(seed, 1, stream)
    xstar = rng.uniform(lo, hi, size=n)
    if kind == SPHERE:
        return ProblemInstance(kind, n, xstar)
    Q = haar_orthogonal(n, rng)
    lamdiag = ellipsoid_diag(n, cond) if kind == ELLIPSOID else None
    return ProblemInstance(kind, n, xstar, Q, lamdiag)


@dataclass
class SearchSpec:
    n: int
    lam: int
    sigma0: float
    x0: np.ndarray
    problem: ProblemInstance


@dataclass
class Workload:
    name: str
    searches: List[SearchSpec]
    box_lo: float
    box_hi: float
    f_target: float
    max_restarts: int
    ipop_double: bool
    generations: int
    notes: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def candidates_per_generation(self):
        return sum(s.lam for s in self.searches)


def start_point(n, lo, hi, seed, stream):
    return rng_for(seed, 2, stream).uniform(lo, hi, size=n)


def ellipsoid_n10(seed=SEED):
    """Plain CMA-ES, no restarts: n=10, lambda=10, sigma0=0.5, x0 ~ U[-4,4]^10,
    rotated ellipsoid with cond 1e6; 2000 generations; stop at f < 1e-10."""
    n = 10
    prob = make_problem(ELLIPSOID, n, seed, 0, cond=1e6)
    x0 = start_point(n, -4.0, 4.0, seed, 0)
    return Workload("ellipsoid-n10-lam10", [SearchSpec(n, 10, 0.5, x0, prob)],
                    -4.0, 4.0, 1e-10, 0, False, 2000)


def rastrigin_n100_ipop(seed=SEED, concurrent=True, levels=10):
    """IPOP on a rotated Rastrigin, n=100, lambda0=17 doubling over 9
    restarts (lambda up to 8704); x* ~ U[-4,4], x0 ~ U[-5,5], sigma0 = 2.5.

    concurrent=True lays the ten population levels 17 * 2^k (k = 0..9) side
    by side as one batch, each level restarting at its own size: the
    K-Distributed layout of the paper's §3.2.3. concurrent=False is the
    sequential IPOP of Algorithm 2 (one search, lambda doubling per restart).
    """
    n = 100
    prob = make_problem(RASTRIGIN, n, seed, 1)
    lam0 = default_lambda(n)
    if concurrent:
        searches = [SearchSpec(n, lam0 << k, 2.5, start_point(n, -5.0, 5.0, seed, 100 + k), prob)
                    for k in range(levels)]
        return Workload("rastrigin-n100-kdist-lam17x2^0..9", searches, -5.0, 5.0,
                        1e-8, 1 << 20, False, 0,
                        notes="K-Distributed: levels lambda=17*2^k run concurrently")
    x0 = start_point(n, -5.0, 5.0, seed, 100)
    return Workload("rastrigin-n100-ipop-lam17", [SearchSpec(n, lam0, 2.5, x0, prob)],
                    -5.0, 5.0, 1e-8, 9, True, 0)


def ellipsoid_n1000(seed=SEED):
    """Single large search: n=1000, lambda=1024, rotated ellipsoid cond 1e6."""
    n = 1000
    prob = make_problem(ELLIPSOID, n, seed, 2, cond=1e6)
    x0 = start_point(n, -4.0, 4.0, seed, 200)
    return Workload("ellipsoid-n1000-lam1024", [SearchSpec(n, 1024, 2.0, x0, prob)],
                    -4.0, 4.0, 1e-8, 0, False, 5000)


def batch256_shapes(seed=SEED, count=256):
    """(n, lambda, objective kind) of every search of the 256-search batch:
    n in {50,200,500,1000,2000} drawn from the seed, lambda = (4 + floor(3 ln
    n)) 2^k with k ~ U{0..8}; objectives alternate rotated ellipsoid and
    rotated Rastrigin by search index."""
    rng = rng_for(seed, 3, 0)
    dims = [50, 200, 500, 1000, 2000]
    shapes = []
    for s in range(count):
        n = int(dims[rng.integers(0, len(dims))])
        k = int(rng.integers(0, 9))
        shapes.append((n, default_lambda(n) << k, ELLIPSOID if s % 2 == 0 else RASTRIGIN))
    return shapes


def batch256(seed=SEED, count=256):
    """Batched concurrent IPOP: the shapes of batch256_shapes, ellipsoids with
    cond 1e6, x0 ~ U[-4,4]^n, sigma0 = 2. Every search restarts at its own
    population size when it stops (the K-Distributed layout of §3.2.3: the
    levels k = 0..8 already run side by side)."""
    searches = []
    for s, (n, lam, kind) in enumerate(batch256_shapes(seed, count)):
        prob = make_problem(kind, n, seed, 1000 + s, cond=1e6)
        searches.append(SearchSpec(n, lam, 2.0, start_point(n, -4.0, 4.0, seed, 1000 + s), prob))
    return Workload("batch256-n50..2000", searches, -4.0, 4.0, 1e-8, 255, False, 0,
                    notes="K-Distributed: 256 searches of uneven (n, lambda) in one batch")


def batch32(seed=SEED):
    """The first 32 searches of the 256-search batch (the same shapes, problems
    and starts): a case small enough for detailed counter captures whose
    eigensolver matrices (144 MB) still exceed the GPU's L2."""
    wl = batch256(seed, count=32)
    wl.name = "batch256-first32"
    return wl


def ellipsoid_n4096(seed=SEED, kind=ELLIPSOID):
    """Large scale: n=4096, lambda=8192, rotated ellipsoid cond 1e4 (or the
    separable sphere control)."""
    n = 4096
    prob = make_problem(kind, n, seed, 4, cond=1e4)
    x0 = start_point(n, -4.0, 4.0, seed, 400)
    return Workload("ellipsoid-n4096-lam8192", [SearchSpec(n, 8192, 2.0, x0, prob)],
                    -4.0, 4.0, 1e-8, 0, False, 2000)


def random_state(n, seed, stream, cond=1e3):
    """A valid mid-run state for teacher-forced checks: SPD C with a known
    eigendecomposition, nonzero paths, a moderate step size."""
    rng = rng_for(seed, 5, stream)
    Bm = haar_orthogonal(n, rng)
    d2 = cond ** rng.uniform(0.0, 1.0, size=n)
    C = (Bm * d2[None, :]) @ Bm.T
    C = 0.5 * (C + C.T)
    return dict(m=rng.uniform(-2.0, 2.0, size=n), sigma=float(rng.uniform(0.05, 0.5)),
                C=C, B=Bm, D=np.sqrt(d2), ps=rng.standard_normal(n) * 0.5,
                pc=rng.standard_normal(n) * 0.1)

"""FP64 CPU oracle for the batched IPOP-CMA-ES generation loop.

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, readable restatement of
the method in "Massively parallel CMA-ES with increasing population" (Redon,
Fortin, Derbel, Tsuji, Sato; arXiv 2409.11765): Algorithm 1 (one CMA-ES
iteration), Eq. (1) (sampling), Eq. (2)/(3) (covariance adaptation) and
Algorithm 2 (IPOP restarts with lambda doubling). Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and
``--impl reference`` arm) may import it. The CUDA engine never imports, links or
calls anything here, and nothing here imports the engine: the two share no code.

Modules
-------
philox    Philox4x32-10 counter-based generator (Salmon et al., SC'11) and the
          Box-Muller normal transform; the random numbers the method draws.
params    strategy parameters as functions of (n, lambda).
cmaes     one generation (sample, evaluate, rank, recombine, cumulate, adapt C,
          step size, lazy eigendecomposition), stop tests and the IPOP restart.
objectives the synthetic objectives (rotated ellipsoid, rotated Rastrigin,
          separable sphere) evaluated in FP64.

Every function is pinned by a ``-m "not gpu"`` test in ``tests/test_oracle_*.py``
against a closed form, an invariant, a hand derivation or a brute force.
"""

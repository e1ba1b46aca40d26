"""One IPOP-CMA-ES generation in plain FP64 (oracle side).

Test infrastructure: see the package docstring.

The steps follow the paper's §2 in its order and notation:

  Algorithm 1, lines 4-6 / Eq. (1)   x_k = m + sigma B D z_k,  z_k ~ N(0, I)
  Algorithm 1, lines 7-9             f_k = f(x_k)
  Algorithm 1, line 10 / §2.1        update (m, C, sigma, p_sigma, p_c):
      rank by f (better points get larger weights w_rk(i), sum one),
      m moved by the weighted selected steps, the paths p_sigma and p_c
      accumulate recent shifts, sigma grows when p_sigma is long and shrinks
      when it is short, and Eq. (2) adapts C:
      C <- C + c_mu sum_i w_rk(i) (y_i y_i^T - C) + c_1 (p_c p_c^T - C)
  §2.1                                B, D from the eigendecomposition of C,
      O(n^3), done lazily every g_eig generations (LAPACK's symmetric eig
      here, the routine the paper calls in §3.1).
  Algorithm 2                         restart with lambda doubled when a stop
      criterion fires (quality not improving, locally flat, distribution too
      small: §2.2).

Where the paper leaves a formula open the reading is the one stated in
params.py and in the comments below (tutorial defaults; the h_sigma stall of
p_c; stop constants after Auger & Hansen 2005).
"""
import math
from dataclasses import dataclass, field

import numpy as np

from . import objectives, philox
from .params import Params

STOP_FTARGET = 1
STOP_MAXITER = 2
STOP_TOLHISTFUN = 4
STOP_TOLX = 8
STOP_CONDITIONCOV = 16
STOP_NOEFFECTAXIS = 32
STOP_NOEFFECTCOORD = 64
STOP_NONFINITE = 128
STOP_ALL = 255

# PD guard after each eigendecomposition: eigenvalues below max * PD_FLOOR are
# lifted to that floor (C and D^2 shifted by the same amount).
PD_FLOOR = 1e-16


@dataclass
class Options:
    f_target: float = -math.inf
    box_lo: float = -4.0
    box_hi: float = 4.0
    max_restarts: int = 9          # descents after the first one
    ipop_double: bool = True       # Algorithm 2: lambda <- 2 lambda per restart
    eig_every: int = 0             # 0: lazy rule of Params.g_eig
    max_iter: int = 0              # 0: Params.max_iter
    tol_hist_fun: float = 1e-12
    tol_x_factor: float = 1e-12    # TolX = factor * sigma0
    cond_max: float = 1e14
    stop_mask: int = STOP_ALL


@dataclass
class State:
    """State of one search (the quantities of Algorithm 1, line 1)."""
    n: int
    lam: int
    sigma: float
    m: np.ndarray
    sigma0: float
    ps: np.ndarray = None
    pc: np.ndarray = None
    C: np.ndarray = None
    B: np.ndarray = None
    D: np.ndarray = None
    gen: int = 0
    restart: int = 0
    best_f: float = math.inf
    best_x: np.ndarray = None
    hist: list = field(default_factory=list)
    done: bool = False
    flags: int = 0

    def __post_init__(self):
        n = self.n
        self.m = np.array(self.m, dtype=np.float64)
        if self.ps is None:
            self.ps = np.zeros(n)
        if self.pc is None:
            self.pc = np.zeros(n)
        if self.C is None:
            self.C = np.eye(n)
        if self.B is None:
            self.B = np.eye(n)
        if self.D is None:
            self.D = np.ones(n)
        if self.best_x is None:
            self.best_x = np.full(n, np.nan)

    def copy(self):
        return State(self.n, self.lam, self.sigma, self.m.copy(), self.sigma0,
                     self.ps.copy(), self.pc.copy(), self.C.copy(), self.B.copy(),
                     self.D.copy(), self.gen, self.restart, self.best_f,
                     self.best_x.copy(), list(self.hist), self.done, self.flags)


@dataclass
class Problem:
    kind: int
    xstar: np.ndarray
    Q: np.ndarray = None
    lamdiag: np.ndarray = None

    def __call__(self, X):
        return objectives.evaluate(self.kind, X, self.Q, self.lamdiag, self.xstar)


def sample(st, Z):
    """Eq. (1) for all candidates at once (the GEMM form of §3.1):
    Y = B D Z, X = m 1^T + sigma Y."""
    Y = st.B @ (st.D[:, None] * Z)
    X = st.m[:, None] + st.sigma * Y
    return Y, X


def rank_order(f):
    """Candidate indices by ascending f; NaN counts as +inf, ties by index."""
    f = np.asarray(f, dtype=np.float64)
    key = np.where(np.isnan(f), np.inf, f)
    return np.lexsort((np.arange(f.shape[0]), key))


def update(st, prm, Z, Y, X, f):
    """Algorithm 1, line 10: update (m, C, sigma, p_sigma, p_c) in place.

    Returns a record of the intermediate quantities for inspection.
    """
    n = st.n
    order = rank_order(f)
    sel = order[:prm.mu]
    w = prm.weights
    yw = Y[:, sel] @ w                      # <y>_w
    zw = Z[:, sel] @ w                      # <z>_w
    sigma_old = st.sigma
    # mean: moved by the fitness-weighted steps (learning rate one)
    st.m = st.m + sigma_old * yw
    # p_sigma: path of recent mean shifts in the isotropic frame, B<z>_w =
    # C^(-1/2) <y>_w with the B, D that produced this generation's points.
    st.ps = ((1.0 - prm.cs) * st.ps
             + math.sqrt(prm.cs * (2.0 - prm.cs) * prm.mueff) * (st.B @ zw))
    psn = float(np.linalg.norm(st.ps))
    # stall of p_c while ||p_sigma|| is large (tutorial's h_sigma)
    hs_lhs = psn / math.sqrt(1.0 - (1.0 - prm.cs) ** (2 * (st.gen + 1)))
    hsig = 1.0 if hs_lhs < (1.4 + 2.0 / (n + 1.0)) * prm.chin else 0.0
    st.pc = ((1.0 - prm.cc) * st.pc
             + hsig * math.sqrt(prm.cc * (2.0 - prm.cc) * prm.mueff) * yw)
    # Eq. (2) in the rewritten form of §3.1 / Eq. (3): since the weights sum to
    # one, C <- (1 - c1 - cmu) C + cmu A.B + c1 p_c p_c^T, with A = [y_i] and
    # B = [w_i y_i^T] over the selected points, plus the h_sigma correction.
    Ysel = Y[:, sel]
    rank_mu = (Ysel * w[None, :]) @ Ysel.T
    delta = (1.0 - hsig) * prm.cc * (2.0 - prm.cc)
    st.C = ((1.0 - prm.c1 - prm.cmu) * st.C
            + prm.c1 * (np.outer(st.pc, st.pc) + delta * st.C)
            + prm.cmu * rank_mu)
    # step size: longer than expected path -> increase, shorter -> decrease
    st.sigma = sigma_old * math.exp((prm.cs / prm.ds) * (psn / prm.chin - 1.0))
    # best sampled point (Algorithm 1, line 12)
    i0 = int(order[0])
    fbest_gen = float(f[i0])
    if fbest_gen < st.best_f:
        st.best_f = fbest_gen
        st.best_x = X[:, i0].copy()
    st.hist.append(fbest_gen)
    if len(st.hist) > prm.hist_len:
        del st.hist[:len(st.hist) - prm.hist_len]
    st.gen += 1
    return dict(order=order, yw=yw, zw=zw, psnorm=psn, hsig=hsig)


def eig_due(st, prm, opts):
    every = opts.eig_every if opts.eig_every > 0 else prm.g_eig
    return st.gen % every == 0


def canonical_basis(B):
    """Sign convention of the eigenvectors: §2.1 only asks for orthonormal
    eigenvectors, so the representative is fixed by making each column's
    entry of largest magnitude (the first on ties) positive. Columns come in
    ascending eigenvalue order from the solver."""
    B = B.copy()
    idx = np.argmax(np.abs(B), axis=0)
    sign = np.where(B[idx, np.arange(B.shape[1])] < 0.0, -1.0, 1.0)
    return B * sign[None, :]


def eig_step(st):
    """B, D from the eigendecomposition of C (§2.1), with a PD guard; columns
    in ascending eigenvalue order with the sign of canonical_basis."""
    n = st.n
    C = 0.5 * (st.C + st.C.T)
    evals, evecs = np.linalg.eigh(C)
    lo = float(evals.min())
    hi = float(evals.max())
    if lo < hi * PD_FLOOR:
        add = hi * PD_FLOOR - lo
        C = C + add * np.eye(n)
        evals = evals + add
    st.C = C
    st.B = canonical_basis(evecs)
    st.D = np.sqrt(evals)


def stop_flags(st, prm, opts):
    """Stop tests of §2.2 (categories from the paper, constants after
    Auger & Hansen 2005): returns a bit mask of the criteria that fire."""
    flags = 0
    n = st.n
    if st.best_f < opts.f_target:
        flags |= STOP_FTARGET
    max_iter = opts.max_iter if opts.max_iter > 0 else prm.max_iter
    if st.gen >= max_iter:
        flags |= STOP_MAXITER
    if len(st.hist) >= prm.hist_len:
        if max(st.hist) - min(st.hist) < opts.tol_hist_fun:
            flags |= STOP_TOLHISTFUN
    diagC = np.diag(st.C)
    tolx = opts.tol_x_factor * st.sigma0
    if np.all(st.sigma * np.abs(st.pc) < tolx) and \
            np.all(st.sigma * np.sqrt(np.maximum(diagC, 0.0)) < tolx):
        flags |= STOP_TOLX
    dmax = float(st.D.max())
    dmin = float(st.D.min())
    if dmax * dmax > opts.cond_max * dmin * dmin:
        flags |= STOP_CONDITIONCOV
    j = st.gen % n
    shift = (0.1 * st.sigma * st.D[j]) * st.B[:, j]
    if np.all(st.m + shift == st.m):
        flags |= STOP_NOEFFECTAXIS
    if np.any(st.m + 0.2 * st.sigma * np.sqrt(np.maximum(diagC, 0.0)) == st.m):
        flags |= STOP_NOEFFECTCOORD
    if not (np.all(np.isfinite(st.m)) and math.isfinite(st.sigma)
            and np.all(np.isfinite(diagC))):
        flags |= STOP_NONFINITE
    return flags & opts.stop_mask


def restart(st, seed, search, opts):
    """Algorithm 2: a new descent with lambda doubled (or kept, for the
    concurrent K-Distributed layout of §3.2.3) and a fresh state."""
    st.restart += 1
    if opts.ipop_double:
        st.lam *= 2
    n = st.n
    st.m = philox.restart_mean(seed, search, st.restart, n, opts.box_lo, opts.box_hi)
    st.sigma = st.sigma0
    st.ps = np.zeros(n)
    st.pc = np.zeros(n)
    st.C = np.eye(n)
    st.B = np.eye(n)
    st.D = np.ones(n)
    st.gen = 0
    st.hist = []


def generation(st, seed, search, problem, opts, Z=None, f=None):
    """One CMA-ES iteration of Algorithm 1 (lines 4-10), the lazy
    eigendecomposition, the stop tests and, when one fires, Algorithm 2's
    restart. Returns a record with Z, Y, X, f and the update intermediates."""
    if st.done:
        return None
    prm = Params(st.n, st.lam)
    if Z is None:
        Z = philox.normals(seed, search, st.restart, st.gen, st.n, st.lam)
    Y, X = sample(st, Z)
    if f is None:
        f = problem(X)
    rec = update(st, prm, Z, Y, X, f)
    rec.update(Z=Z, Y=Y, X=X, f=np.asarray(f, dtype=np.float64))
    rec["eig"] = eig_due(st, prm, opts)
    if rec["eig"]:
        eig_step(st)
    flags = stop_flags(st, prm, opts)
    st.flags = flags
    rec["flags"] = flags
    if flags:
        if (flags & STOP_FTARGET) or st.restart + 1 > opts.max_restarts:
            st.done = True
        else:
            restart(st, seed, search, opts)
    return rec


def run(st, seed, search, problem, opts, generations):
    """Run up to `generations` generations (fewer if the search finishes)."""
    done = 0
    while done < generations and not st.done:
        generation(st, seed, search, problem, opts)
        done += 1
    return done

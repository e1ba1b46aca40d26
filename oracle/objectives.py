"""Synthetic objectives evaluated in FP64 (oracle side).

Test infrastructure: see the package docstring.

The paper treats f as a black box (§1, Algorithm 1) and benchmarks on BBOB
(§4.1). Seeded synthetic stand-ins of the same families are used instead:

  rotated ellipsoid   f(x) = sum_i Lambda_i u_i^2,             u = Q (x - x*)
  rotated Rastrigin   f(x) = 10 n + sum_i (u_i^2 - 10 cos(2 pi u_i))
  separable sphere    f(x) = sum_i (x_i - x*_i)^2

X holds one candidate per column (n x lam).
"""
import numpy as np

ELLIPSOID = 1
RASTRIGIN = 2
SPHERE = 3


def rotate(X, Q, xstar):
    """u = Q (x - x*) for every column of X."""
    return Q @ (X - xstar[:, None])


def ellipsoid(X, Q, lamdiag, xstar):
    U = rotate(X, Q, xstar)
    return np.sum(lamdiag[:, None] * U * U, axis=0)


def rastrigin(X, Q, xstar):
    U = rotate(X, Q, xstar)
    n = X.shape[0]
    return 10.0 * n + np.sum(U * U - 10.0 * np.cos((2.0 * np.pi) * U), axis=0)


def sphere(X, xstar):
    R = X - xstar[:, None]
    return np.sum(R * R, axis=0)


def evaluate(kind, X, Q=None, lamdiag=None, xstar=None):
    if kind == ELLIPSOID:
        return ellipsoid(X, Q, lamdiag, xstar)
    if kind == RASTRIGIN:
        return rastrigin(X, Q, xstar)
    if kind == SPHERE:
        return sphere(X, xstar)
    raise ValueError("unknown objective kind %r" % (kind,))


def magnitude(kind, X, Q=None, lamdiag=None, xstar=None):
    """Sum of the absolute terms of f: the scale of its rounding error."""
    if kind == ELLIPSOID:
        U = rotate(X, Q, xstar)
        return np.sum(np.abs(lamdiag[:, None]) * U * U, axis=0)
    if kind == RASTRIGIN:
        U = rotate(X, Q, xstar)
        return 10.0 * X.shape[0] + np.sum(U * U + 10.0, axis=0)
    return sphere(X, xstar)

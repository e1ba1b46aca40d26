"""Pins for the strategy parameters (the reading of §2.1's open defaults)."""
import math

import numpy as np
import pytest
from scipy.special import gammaln

from oracle.params import Params, default_lambda, expected_norm


@pytest.mark.parametrize("n,lam", [(2, 6), (10, 10), (50, 15), (100, 17), (200, 19),
                                   (500, 22), (1000, 24), (2000, 26), (4096, 28)])
def test_default_lambda_table(n, lam):
    assert default_lambda(n) == lam


@pytest.mark.parametrize("n,lam", [(2, 6), (10, 10), (100, 17), (100, 8704), (1000, 1024),
                                   (4096, 8192), (3, 3), (5, 2)])
def test_weights_sum_to_one_and_decrease(n, lam):
    p = Params(n, lam)
    assert p.mu == lam // 2
    assert abs(p.weights.sum() - 1.0) < 1e-15 * max(1, p.mu) ** 0.5 * 4
    assert np.all(p.weights > 0)
    assert np.all(np.diff(p.weights) < 0) or p.mu == 1
    assert 1.0 - 1e-12 <= p.mueff <= p.mu + 1e-9
    # mu_eff = (sum w')^2 / sum w'^2 for the unnormalised log weights
    wp = np.array([math.log((lam + 1) / 2.0) - math.log(i) for i in range(1, p.mu + 1)])
    assert math.isclose(p.mueff, wp.sum() ** 2 / (wp ** 2).sum(), rel_tol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 3, 10, 100, 1000, 4096])
def test_expected_norm_vs_exact(n):
    exact = math.sqrt(2.0) * math.exp(gammaln((n + 1) / 2.0) - gammaln(n / 2.0))
    rel = abs(expected_norm(n) - exact) / exact
    # the approximation error is below 1e-3 and falls like n^-2 (about
    # 0.016 / n^2 for large n; 7.6e-4 at n = 2)
    assert rel < 1e-3
    assert rel < 0.02 / n ** 2


def test_learning_rate_ranges():
    for n in (2, 10, 100, 1000, 4096):
        for lam in (default_lambda(n), 4 * default_lambda(n), 1024, 8192):
            p = Params(n, lam)
            assert 0 < p.c1 and 0 <= p.cmu and p.c1 + p.cmu <= 1.0 + 1e-15
            assert 0 < p.cs < 1 and 0 < p.cc <= 1
            assert p.ds >= 1.0
            assert p.g_eig >= 1


def test_n2_lambda6_values_by_hand():
    """Scalar re-derivation for n=2, lambda=6 (mu=3)."""
    n, lam = 2, 6
    wp = [math.log(3.5) - math.log(1), math.log(3.5) - math.log(2), math.log(3.5) - math.log(3)]
    s = wp[0] + wp[1] + wp[2]
    w = [x / s for x in wp]
    mueff = 1.0 / (w[0] ** 2 + w[1] ** 2 + w[2] ** 2)
    p = Params(n, lam)
    assert np.allclose(p.weights, w, rtol=1e-15, atol=0)
    assert math.isclose(p.mueff, mueff, rel_tol=1e-15)
    assert math.isclose(p.c1, 2.0 / (3.3 ** 2 + mueff), rel_tol=1e-15)
    assert math.isclose(p.cmu, 2.0 * (mueff - 2.0 + 1.0 / mueff) / (16.0 + mueff), rel_tol=1e-15)
    assert math.isclose(p.cs, (mueff + 2.0) / (7.0 + mueff), rel_tol=1e-15)
    assert math.isclose(p.cc, (4.0 + mueff / 2.0) / (6.0 + mueff), rel_tol=1e-15)
    assert math.isclose(p.chin, math.sqrt(2.0) * (1.0 - 1.0 / 8.0 + 1.0 / 84.0), rel_tol=1e-15)
    # the same numbers to 12 digits
    assert np.allclose(p.weights, [0.637042571241, 0.284570257438, 0.078387171321], atol=5e-13)
    assert abs(p.mueff - 2.028611464610) < 5e-12
    assert abs(p.c1 - 0.154815399896) < 5e-13
    assert abs(p.cmu - 0.057859085072) < 5e-13
    assert abs(p.cs - 0.446204987378) < 5e-13
    assert abs(p.ds - 1.446204987378) < 5e-13
    assert abs(p.cc - 0.624554539027) < 5e-13
    assert abs(p.chin - 1.254272742819) < 5e-13


def test_lazy_eig_cadence_examples():
    # 1 / ((c1 + cmu) n 10): about 0.28 for n=10, lambda=10; 1.3 for n=100, lambda=17
    assert Params(10, 10).g_eig == 1
    assert Params(100, 17).g_eig == 1
    assert Params(100, 8704).g_eig == 1
    # small populations in high dimension amortise the eigendecomposition
    assert Params(2000, 26).g_eig > 1
    p = Params(2000, 26)
    assert p.g_eig == int(math.floor(1.0 / ((p.c1 + p.cmu) * 2000 * 10)))

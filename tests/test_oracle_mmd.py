"""Pins of the MMD oracle (CPU only): closed forms, the population limit
for Gaussian clouds, invariances and central differences of its gradient."""
import math

import numpy as np
import pytest

from oracle import mmd


def test_single_points_closed_form():
    """One point each: MMD^2 = sum_l [2 - 2 exp(-d^2 / (2 sigma_l^2))];
    with d^2 = 2 (standardised), sigma = 1: 2 - 2/e = 1.2642411176571153,
    sigma = 2: 2 - 2 exp(-1/4) = 0.4423984338571902."""
    a = np.array([[1.0, 2.0, 3.0, 0.0, 0.0, 0.0]])
    s = np.array([2.0, 1.0, 1.0, 3.0, 1.0, 1.0])
    b = a + np.array([[2.0, 1.0, 0.0, 0.0, 0.0, 0.0]])  # d^2 = 1 + 1 = 2
    mu = np.zeros(6)
    assert mmd.mmd2(a, b, [1.0], mu, s) == pytest.approx(1.2642411176571153, rel=1e-14)
    assert mmd.mmd2(a, b, [1.0, 2.0], mu, s) == pytest.approx(
        1.2642411176571153 + 0.4423984338571902, rel=1e-14)


def test_identical_clouds_and_nonnegativity():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(40, 6))
    assert abs(mmd.mmd2(X, X, [0.5, 1.0, 2.0])) < 1e-13
    for k in range(5):
        Y = rng.normal(size=(30, 6)) * rng.uniform(0.5, 2.0) + rng.normal(size=6)
        assert mmd.mmd2(X, Y, [0.7, 1.5]) > 0.0


def test_gaussian_population_limit():
    """X ~ N(0, I_6), Y ~ N(delta, I_6), sigma = 2, fixed standardisation:
    E k(x, x') = (s2/(s2+2))^3 = A, E k(x, y) = A exp(-|delta|^2/(2 (s2+2))),
    and the V-statistic has mean 1/n + (1-1/n) A + 1/m + (1-1/m) A
    - 2 A exp(-|delta|^2/12).  n = m = 1500 (sampling error about 1 %)."""
    rng = np.random.default_rng(1)
    n = m = 1500
    delta = np.array([3.0, 0, 0, 0, 0, 0])
    X = rng.normal(size=(n, 6))
    Y = rng.normal(size=(m, 6)) + delta
    A = (4.0 / 6.0) ** 3
    expect = 1 / n + (1 - 1 / n) * A + 1 / m + (1 - 1 / m) * A - 2 * A * math.exp(-9.0 / 12.0)
    got = mmd.mmd2(X, Y, [2.0], np.zeros(6), np.ones(6))
    assert got == pytest.approx(expect, rel=0.05)


def test_invariances():
    """Standardised by the target's statistics, MMD^2 is unchanged by a common
    shift or per-dimension scaling of both clouds and by reordering."""
    rng = np.random.default_rng(2)
    X = rng.normal(size=(25, 6))
    Y = rng.normal(size=(33, 6)) * 1.3 + 0.4
    base = mmd.mmd2(X, Y, [0.5, 1.0])
    sh = rng.normal(size=6) * 10
    sc = rng.uniform(0.1, 10.0, size=6)
    assert mmd.mmd2(X * sc + sh, Y * sc + sh, [0.5, 1.0]) == pytest.approx(base, rel=1e-11)
    assert mmd.mmd2(X[::-1], Y[rng.permutation(33)], [0.5, 1.0]) == pytest.approx(base, rel=1e-12)


def test_gradient_central_differences():
    rng = np.random.default_rng(3)
    X = rng.normal(size=(7, 6))
    Y = rng.normal(size=(9, 6)) + 0.3
    mu, s = mmd.target_stats(Y)
    sig = [0.6, 1.7]
    L, g = mmd.mmd2_grad(X, Y, sig, mu, s)
    assert L == pytest.approx(mmd.mmd2(X, Y, sig, mu, s), rel=1e-14)
    for (i, d) in ((0, 0), (3, 2), (6, 5), (2, 4)):
        def f(h):
            Z = X.copy()
            Z[i, d] += h
            return mmd.mmd2(Z, Y, sig, mu, s)
        h = 1e-4
        fd = (f(h) - f(-h)) / (2 * h)
        fd2 = (f(h / 2) - f(-h / 2)) / h
        assert (4 * fd2 - fd) / 3 == pytest.approx(g[i, d], rel=1e-8, abs=1e-12)

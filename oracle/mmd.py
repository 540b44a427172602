"""Maximum mean discrepancy between phase-space point clouds, FP64 numpy.

TEST INFRASTRUCTURE ONLY.

The paper's first inference method (Sec. 2.2.1; Fig. 2, step 4) treats the
simulated and the observed stream as point clouds and compares them with the
maximum mean discrepancy; the grid search of that method ranks 10^4
parameter vectors by it.  The paper names neither the kernel nor its
bandwidth.  Readings used here:

  * a point is q = (x, y, z, vx, vy, vz), Galactocentric position and
    velocity (the paper uses the full 6D phase-space information);
  * coordinates are standardised per dimension, u = (q - mu) / s, with mu
    and s the mean and standard deviation of the target cloud unless given
    (fixed numbers: they are not differentiated);
  * the kernel is a sum of Gaussians over a few bandwidths,
    k(a, b) = sum_l exp(-|u_a - u_b|^2 / (2 sigma_l^2));
  * the estimator is the biased one (a V-statistic, self-pairs included),
    MMD^2 = 1/n^2 sum_{i,i'} k(x_i, x_i') + 1/m^2 sum_{j,j'} k(y_j, y_j')
            - 2/(n m) sum_{i,j} k(x_i, y_j).

Every function is the definition written out with numpy broadcasting; the
gradient is the derivative of that definition by hand:
  d MMD^2 / d u_i = 2/n [ 1/n sum_i' g(x_i, x_i') - 1/m sum_j g(x_i, y_j) ],
  g(a, b) = d k(a, b) / d u_a = sum_l exp(-|u_a - u_b|^2 / (2 sigma_l^2))
                                 (u_b - u_a) / sigma_l^2,
and d/dq = (d/du) / s.
"""
from __future__ import annotations

import numpy as np


def target_stats(Y):
    """Per-dimension mean and standard deviation of a cloud (m, 6)."""
    Y = np.asarray(Y, float)
    return Y.mean(axis=0), Y.std(axis=0)


def gram_sum(A, B, sigmas, rows=256):
    """sum_{a, b} k(A_a, B_b), k(a, b) = sum_l exp(-|a - b|^2 / (2 sigma_l^2)),
    for standardised points A (p, d), B (q, d); rows of A in blocks."""
    tot = 0.0
    for r0 in range(0, A.shape[0], rows):
        d2 = np.sum((A[r0:r0 + rows, None, :] - B[None, :, :]) ** 2, axis=2)
        tot += sum(np.exp(-d2 / (2.0 * s * s)) for s in sigmas).sum()
    return tot


def _kgrad_sum(A, B, sigmas, rows=512):
    """G[a] = sum_b g(A_a, B_b) with g the kernel's gradient in its first
    argument (see the module docstring); rows of A in blocks."""
    out = np.zeros_like(A)
    for r0 in range(0, A.shape[0], rows):
        a = A[r0:r0 + rows]
        D = B[None, :, :] - a[:, None, :]            # u_b - u_a
        d2 = np.sum(D * D, axis=2)
        c = sum(np.exp(-d2 / (2.0 * s * s)) / (s * s) for s in sigmas)
        out[r0:r0 + rows] = np.einsum("ab,abk->ak", c, D)
    return out


def mmd2(X, Y, sigmas, mu=None, s=None):
    """Biased MMD^2 between clouds X (n, 6) and Y (m, 6)."""
    X = np.asarray(X, float)
    Y = np.asarray(Y, float)
    if mu is None or s is None:
        mu, s = target_stats(Y)
    U = (X - mu) / s
    V = (Y - mu) / s
    n, m = len(U), len(V)
    return (gram_sum(U, U, sigmas) / (n * n) + gram_sum(V, V, sigmas) / (m * m)
            - 2.0 * gram_sum(U, V, sigmas) / (n * m))


def mmd2_grad(X, Y, sigmas, mu=None, s=None):
    """(MMD^2, dMMD^2/dX) with the gradient shaped like X (n, 6)."""
    X = np.asarray(X, float)
    Y = np.asarray(Y, float)
    if mu is None or s is None:
        mu, s = target_stats(Y)
    U = (X - mu) / s
    V = (Y - mu) / s
    n, m = len(U), len(V)
    L = mmd2(X, Y, sigmas, mu, s)
    gu = (2.0 / n) * (_kgrad_sum(U, U, sigmas) / n - _kgrad_sum(U, V, sigmas) / m)
    return L, gu / s


def cloud(x, v):
    """(n, 3) positions and velocities -> (n, 6) phase-space points."""
    return np.concatenate([np.asarray(x, float), np.asarray(v, float)], axis=1)

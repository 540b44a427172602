"""Seeded synthetic inputs for the N-body workloads.

This module is the one piece shared by the CUDA path's callers and by the
FP64 oracle's tests: it draws the random initial conditions and nothing
else.  It holds none of the method's arithmetic (no forces, no integrator,
no gradients, no stream head).

Plummer sphere sampling follows the classical recipe of Aarseth, Henon and
Wielen (1974): radius from the inverse of the enclosed-mass fraction
M(<r)/M = r^3 / (1 + r^2)^(3/2), speed by von Neumann rejection from
g(q) = q^2 (1 - q^2)^(7/2) with v = q * sqrt(2) * (1 + r^2)^(-1/4), isotropic
directions, then the centre of mass and its velocity are removed.  The paper
samples its progenitor from an equilibrium Plummer sphere (Fig. 2, step 3;
Sec. 2.2.1).  Samples are drawn in the unit model G = M = a = 1.
"""
from __future__ import annotations

import numpy as np


def _isotropic(rng: np.random.Generator, n: int) -> np.ndarray:
    cos_t = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    sin_t = np.sqrt(1.0 - cos_t * cos_t)
    return np.stack([sin_t * np.cos(phi), sin_t * np.sin(phi), cos_t], axis=1)


def plummer_unit(n: int, seed: int, rmax: float = 10.0):
    """Equal-mass Plummer sphere in the unit model (G = M = a = 1).

    Returns (xhat, vhat), each float64 of shape (n, 3), centre of mass and
    mean velocity exactly removed.  Radii beyond rmax are redrawn (the model
    is truncated at 10 scale radii, 99.1 % of its mass)."""
    if n <= 0:
        return np.zeros((0, 3)), np.zeros((0, 3))
    rng = np.random.default_rng(seed)
    r = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        X1 = rng.uniform(0.0, 1.0, todo.size)
        X1 = np.where(X1 == 0.0, 0.5, X1)
        rr = 1.0 / np.sqrt(X1 ** (-2.0 / 3.0) - 1.0)
        ok = rr <= rmax
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    x = r[:, None] * _isotropic(rng, n)

    q = np.empty(n)
    todo = np.arange(n)
    while todo.size:
        X4 = rng.uniform(0.0, 1.0, todo.size)
        X5 = rng.uniform(0.0, 1.0, todo.size)
        ok = 0.1 * X5 < X4 * X4 * (1.0 - X4 * X4) ** 3.5
        q[todo[ok]] = X4[ok]
        todo = todo[~ok]
    speed = q * np.sqrt(2.0) * (1.0 + r * r) ** (-0.25)
    v = speed[:, None] * _isotropic(rng, n)

    x -= x.mean(axis=0)
    v -= v.mean(axis=0)
    return x, v


def plummer_sphere(n: int, seed: int, G: float, M: float, a: float,
                   center=(0.0, 0.0, 0.0), velocity=(0.0, 0.0, 0.0)):
    """A Plummer sphere of total mass M and scale radius a placed at
    (center, velocity): input recipe of the fixed-parameter workloads.

    Returns (x, v, m): (n, 3), (n, 3), (n,) float64."""
    xh, vh = plummer_unit(n, seed)
    vscale = np.sqrt(G * M / a)
    x = a * xh + np.asarray(center, dtype=np.float64)
    v = vscale * vh + np.asarray(velocity, dtype=np.float64)
    m = np.full(n, M / n)
    return x, v, m


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Simulation sizes drawn log-uniformly in [lo, hi] (ensemble workload)."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(lo), np.log(hi), count))).astype(np.int64)


def uniform_factors(count: int, width: float, dims: int, seed: int) -> np.ndarray:
    """Multiplicative parameter factors drawn uniformly in [1-width, 1+width]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(1.0 - width, 1.0 + width, (count, dims))


def perturbed_clouds(x: np.ndarray, v: np.ndarray, sigma_x: float, sigma_v: float,
                     count: int, seed: int):
    """`count` realisations of an observed cloud (x, v: (n, 3) each) with
    every coordinate drawn from a Gaussian around its observed value:
    standard deviation sigma_x for positions, sigma_v for velocities (the
    bootstrap of the paper's first inference method, Sec. 2.2.1, which
    resamples the observation by its observational errors); sigma_x and
    sigma_v are scalars or per-coordinate (3,) arrays.  Returns (count, n, 3)
    positions and velocities."""
    rng = np.random.default_rng(seed)
    x = np.asarray(x, float)
    v = np.asarray(v, float)
    ex = rng.normal(size=(count,) + x.shape) * sigma_x
    ev = rng.normal(size=(count,) + v.shape) * sigma_v
    return x[None] + ex, v[None] + ev

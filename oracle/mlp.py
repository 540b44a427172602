"""FP64 reference of the density surrogate (TEST INFRASTRUCTURE ONLY).

The paper names coupling the simulator with a neural network as future work
(Sec. 3).  The surrogate here maps the four physical parameters (normalised)
to the 32 x 32 binned stream density:

    h1 = GELU(W1 u + b1),  h2 = GELU(W2 h1 + b2),  y = W3 h2 + b3,

GELU(z) = z Phi(z) with the exact normal CDF Phi, loss = mean squared error
over the batch and the outputs, optimiser Adam (Kingma & Ba 2015) with bias
correction.  Weights are stored out x in (row-major), like a linear layer.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(params, u):
    """Returns y and the cache of pre-activations needed by backward."""
    W1, b1, W2, b2, W3, b3 = params
    z1 = u @ W1.T + b1
    h1 = gelu(z1)
    z2 = h1 @ W2.T + b2
    h2 = gelu(z2)
    y = h2 @ W3.T + b3
    return y, (u, z1, h1, z2, h2)


def mse(y, t):
    return float(np.mean((y - t) ** 2))


def backward(params, cache, y, t):
    """Gradients of mse(y, t) w.r.t. (W1, b1, W2, b2, W3, b3) and u."""
    W1, b1, W2, b2, W3, b3 = params
    u, z1, h1, z2, h2 = cache
    gy = 2.0 * (y - t) / y.size
    gW3 = gy.T @ h2
    gb3 = gy.sum(axis=0)
    gh2 = gy @ W3
    gz2 = gh2 * gelu_grad(z2)
    gW2 = gz2.T @ h1
    gb2 = gz2.sum(axis=0)
    gh1 = gz2 @ W2
    gz1 = gh1 * gelu_grad(z1)
    gW1 = gz1.T @ u
    gb1 = gz1.sum(axis=0)
    gu = gz1 @ W1
    return (gW1, gb1, gW2, gb2, gW3, gb3), gu


def adam_step(w, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns new (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v

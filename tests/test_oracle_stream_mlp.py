"""Pins of the stream-density head, the whole mock-stream pipeline gradient,
the surrogate MLP reference and the Plummer input sampler (CPU only)."""
import dataclasses
import math

import numpy as np
import pytest

from oracle import mlp, stream
from paper_2511_22468_gb300.configs import C1
from paper_2511_22468_gb300.inputs import plummer_unit


# ------------------------------------------------------------------- head --
def test_projection_axes():
    fr = stream.frame(C1.X0, C1.V0, C1.observer)
    e1, e2, n = fr
    obs = np.array(C1.observer)
    pts = np.array([obs + 3 * e1, obs + 2 * e2, obs + 5 * n, obs - 4 * e2,
                    np.array(C1.X0)])
    p1, p2 = stream.project(pts, C1.observer, fr)
    np.testing.assert_allclose(p1[[0, 1, 3, 4]], [0, math.pi / 2, -math.pi / 2, 0], atol=1e-14)
    np.testing.assert_allclose(p2[[0, 1, 2, 3, 4]], [0, 0, math.pi / 2, 0, 0], atol=1e-7)
    # the progenitor moves toward +phi1 (V0 has a positive e2 component)
    assert np.dot(C1.V0, e2) > 0


def test_soft_hist_one_sigma_weights():
    """A particle at a bin centre puts Phi(1) - Phi(-1) = 0.6826894921370859
    of its mass in that bin and Phi(3) - Phi(1) = 0.15730535589982697 in
    each neighbour (sigma is half a bin)."""
    e1 = stream.edges(-90, 90, 32)
    e2 = stream.edges(-10, 10, 32)
    c1 = 0.5 * (e1[10] + e1[11])
    c2 = 0.5 * (e2[20] + e2[21])
    rho = stream.soft_hist(np.array([c1]), np.array([c2]), e1, e2)
    assert rho[10, 20] == pytest.approx(0.6826894921370859 ** 2, rel=1e-12)
    assert rho[11, 20] == pytest.approx(0.15730535589982697 * 0.6826894921370859, rel=1e-10)
    assert rho.sum() == pytest.approx(1.0, abs=1e-12)


def test_head_vjp_vs_fd():
    rng = np.random.default_rng(0)
    fr = stream.frame(C1.X0, C1.V0, C1.observer)
    e1 = stream.edges(-90, 90, 32)
    e2 = stream.edges(-10, 10, 32)
    x = np.array(C1.X0) + rng.normal(size=(50, 3)) * np.array([3, 3, 0.3])
    target = rng.uniform(0, 0.01, (32, 32))

    def L(xx):
        p1, p2 = stream.project(xx, C1.observer, fr)
        return np.mean((stream.soft_hist(p1, p2, e1, e2) - target) ** 2)

    p1, p2 = stream.project(x, C1.observer, fr)
    rho = stream.soft_hist(p1, p2, e1, e2)
    g1, g2 = stream.soft_hist_vjp(p1, p2, e1, e2, 2 * (rho - target) / rho.size)
    xb = stream.project_vjp(x, C1.observer, fr, g1, g2)
    h = 1e-6
    for i, d in ((0, 0), (13, 1), (49, 2), (25, 0)):
        xp, xm = x.copy(), x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        assert (L(xp) - L(xm)) / (2 * h) == pytest.approx(xb[i, d], rel=1e-5, abs=1e-14)


def test_stream_pipeline_gradient_vs_fd():
    """dL/dTheta of the whole pipeline (orbit back, Plummer shift, forward,
    head) against central differences, on a shortened workload that keeps
    the stream workload's dt = 0.5 Myr (a much coarser step makes the
    tangent dynamics of the progenitor blow up)."""
    cfg = dataclasses.replace(C1, n=48, t_acc=30.0, n_steps=60)
    xh, vh = plummer_unit(48, 1)
    model = stream.StreamModel(cfg, xh, vh)
    truth = np.array(cfg.theta_true, float)
    target = model.density(truth)
    th = truth * np.array([1.05, 0.9, 1.1, 0.95])
    L0, g = model.loss_and_grad(th, target)
    assert L0 > 0
    for k in range(4):
        h = 1e-4 * th[k]
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        tp2, tm2 = th.copy(), th.copy()
        tp2[k] += h / 2
        tm2[k] -= h / 2
        d1 = (model.loss(tp, target) - model.loss(tm, target)) / (2 * h)
        d2 = (model.loss(tp2, target) - model.loss(tm2, target)) / h
        assert (4 * d2 - d1) / 3 == pytest.approx(g[k], rel=1e-5)


def test_stream_mmd_pipeline_gradient_vs_fd():
    """The point-cloud (MMD) form of the pipeline: dL/dTheta against central
    differences; the target cloud is the simulated stream at the true
    parameters with the same unit sample, standardised by its own
    statistics (held fixed)."""
    from oracle import mmd
    cfg = dataclasses.replace(C1, n=48, t_acc=30.0, n_steps=60)
    xh, vh = plummer_unit(48, 1)
    model = stream.StreamModel(cfg, xh, vh)
    truth = np.array(cfg.theta_true, float)
    xt, vt = model.final_state(truth)
    Y = mmd.cloud(xt, vt)
    mu, sd = mmd.target_stats(Y)
    sig = [0.5, 1.0, 2.0]
    assert model.mmd_loss(truth, Y, sig, mu, sd) == pytest.approx(0.0, abs=1e-15)
    th = truth * np.array([1.05, 0.9, 1.1, 0.95])
    L0, g = model.mmd_loss_and_grad(th, Y, sig, mu, sd)
    assert L0 > 0
    for k in range(4):
        h = 1e-4 * th[k]
        def f(e):
            t = th.copy()
            t[k] += e
            return model.mmd_loss(t, Y, sig, mu, sd)
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        assert (4 * d2 - d1) / 3 == pytest.approx(g[k], rel=1e-5)
    # the two parts the error bounds use add up to the gradient (recomputed
    # at th: the FD calls above do not touch them)
    model.mmd_loss_and_grad(th, Y, sig, mu, sd)
    p1, p2 = model.grad_parts
    np.testing.assert_allclose(p1 + p2, g, rtol=1e-14, atol=0.0)
    assert p1[0] == model.t_end_parts[0] and p2[0] == model.t_end_parts[1]


def test_stream_loss_zero_at_truth():
    cfg = dataclasses.replace(C1, n=32, t_acc=100.0, n_steps=20)
    xh, vh = plummer_unit(32, 1)
    model = stream.StreamModel(cfg, xh, vh)
    truth = np.array(cfg.theta_true, float)
    L, g = model.loss_and_grad(truth, model.density(truth))
    assert L == 0.0 and np.all(g == 0.0)


# -------------------------------------------------------------------- mlp --
def test_gelu_values():
    """GELU(z) = z Phi(z): Phi(1) = 0.8413447460685429, Phi(-1) = 0.15865525393145707."""
    np.testing.assert_allclose(mlp.gelu(np.array([1.0, -1.0, 0.0])),
                               [0.8413447460685429, -0.15865525393145707, 0.0], rtol=1e-15)
    z = np.linspace(-4, 4, 17)
    np.testing.assert_allclose(mlp.gelu_grad(z), (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6,
                               rtol=1e-7, atol=1e-9)


def _params(rng, din=4, h=16, dout=12):
    return [rng.normal(size=(h, din)) * 0.5, rng.normal(size=h) * 0.1,
            rng.normal(size=(h, h)) * 0.3, rng.normal(size=h) * 0.1,
            rng.normal(size=(dout, h)) * 0.3, rng.normal(size=dout) * 0.1]


def test_mlp_backward_vs_fd():
    rng = np.random.default_rng(1)
    P = _params(rng)
    u = rng.normal(size=(5, 4))
    t = rng.normal(size=(5, 12))
    y, cache = mlp.forward(P, u)
    grads, gu = mlp.backward(P, cache, y, t)
    h = 1e-6
    for pi in range(6):
        flat = P[pi].reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            Pp = [p.copy() for p in P]
            Pm = [p.copy() for p in P]
            Pp[pi].reshape(-1)[idx] += h
            Pm[pi].reshape(-1)[idx] -= h
            fd = (mlp.mse(mlp.forward(Pp, u)[0], t) - mlp.mse(mlp.forward(Pm, u)[0], t)) / (2 * h)
            assert fd == pytest.approx(grads[pi].reshape(-1)[idx], rel=1e-6, abs=1e-10)
    up, um = u.copy(), u.copy()
    up[2, 1] += h
    um[2, 1] -= h
    fd = (mlp.mse(mlp.forward(P, up)[0], t) - mlp.mse(mlp.forward(P, um)[0], t)) / (2 * h)
    assert fd == pytest.approx(gu[2, 1], rel=1e-6)


def test_mlp_tiny_closed_form():
    """One input, one hidden unit per layer, identity-like weights:
    y = w3 GELU(w2 GELU(w1 u + b1) + b2) + b3 by hand."""
    P = [np.array([[2.0]]), np.array([-1.0]), np.array([[1.0]]), np.array([0.0]),
         np.array([[3.0]]), np.array([0.5])]
    y, _ = mlp.forward(P, np.array([[1.0]]))
    h1 = 0.8413447460685429          # GELU(1)
    h2 = h1 * 0.7999225850214973  # GELU(h1) = h1 Phi(h1)
    assert y[0, 0] == pytest.approx(3.0 * h2 + 0.5, rel=1e-9)


def test_adam_first_step():
    """At t = 1 bias correction gives w - lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3])
    w, m, v = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    np.testing.assert_allclose(w, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


# ----------------------------------------------------------------- inputs --
def test_plummer_sampler_profile():
    """Enclosed mass M(<r) = r^3/(1+r^2)^1.5 (KS distance), half-mass radius
    1.305, virial-ratio proxy <v^2> = |W|/M = 3 pi/32 for the untruncated
    model (within sampling noise and the 10 a truncation)."""
    x, v = plummer_unit(20000, 3)
    r = np.sort(np.linalg.norm(x, axis=1))
    cdf_model = r ** 3 / (1 + r * r) ** 1.5 / (1000 / 101 ** 1.5)
    emp = np.arange(1, r.size + 1) / r.size
    assert np.abs(emp - cdf_model).max() < 0.015
    assert np.median(r) == pytest.approx(1.305, rel=0.03)
    assert np.mean(np.sum(v * v, axis=1)) == pytest.approx(3 * math.pi / 32, rel=0.03)
    assert np.abs(x.mean(axis=0)).max() < 1e-14 and np.abs(v.mean(axis=0)).max() < 1e-15


def test_plummer_sampler_seeded():
    a = plummer_unit(100, 7)
    b = plummer_unit(100, 7)
    c = plummer_unit(100, 8)
    assert np.array_equal(a[0], b[0]) and not np.array_equal(a[0], c[0])


def test_golden_stream_n1e4_adjoint_matches_differences():
    """The stored oracle values of the stream pipeline at N = 10^4
    (tests/golden/stream_n1e4_s*.json, written by make_stream_n1e4.py): the
    oracle's adjoint agrees with its own Richardson central differences
    (1e-4 relative per component; dL/dt_end to 1e-4 of its two parts), the
    parts add up to the gradient, the loss is the mean squared difference of
    the stored densities, and the density is normalised (mass fraction of
    the particles inside the window)."""
    import glob
    import json
    import os
    files = sorted(glob.glob(os.path.join(os.path.dirname(__file__), "golden",
                                          "stream_n1e4_s*.json")))
    assert files
    for f in files:
        g = json.load(open(f))
        grad = np.array(g["grad"])
        fd = np.array(g["grad_fd_richardson"])
        p1, p2 = (np.array(p) for p in g["grad_parts"])
        np.testing.assert_allclose(p1 + p2, grad, rtol=1e-12, atol=0)
        scale = np.abs(fd)
        scale[0] = sum(abs(p) for p in g["t_end_parts"])
        assert np.all(np.abs(grad - fd) <= 1e-4 * scale), f
        rho, tgt = np.array(g["density"]), np.array(g["target_density"])
        assert g["loss"] == pytest.approx(np.mean((rho - tgt) ** 2), rel=1e-12)
        assert 0.0 < rho.sum() <= 1.0 and 0.0 < tgt.sum() <= 1.0

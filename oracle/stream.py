"""Stream-density head and the mock-stream pipeline, FP64 numpy oracle.

TEST INFRASTRUCTURE ONLY.

The paper's inference pipeline (Fig. 2; Sec. 2.2.1) takes the progenitor's
present-day centre of mass, integrates it backward as a single particle for
t_end in the external potential, replaces it by a Plummer sphere shifted to
the recovered phase-space point, integrates forward, and compares the
simulated stream with the observed one.  The paper compares point clouds
with an MMD; the workload here compares binned sky densities, with a squared
error loss.  Readings of points the paper leaves open:

  * step count fixed at n; dt = t_end / n (so t_end stays differentiable),
    the backward orbit uses dt_b = -t_end / n with the same n;
  * unit Plummer sample (xhat, vhat) scaled as x = a xhat + X,
    v = sqrt(G M_prog / a) vhat + V, equal masses M_prog / N;
  * sky frame (synthetic; the GD-1 rotation is not used): observer at x_obs,
    e1 = unit(X0 - x_obs), pole n = unit((X0 - x_obs) x V0), e2 = n x e1;
    phi1 = atan2(d.e2, d.e1), phi2 = asin(d.n / |d|), d = x - x_obs;
  * soft histogram: each particle spreads over the bins with Gaussian
    weights of width sigma = half a bin, a bin receiving the normal-CDF mass
    between its edges, rho[b1, b2] = (1/N) sum_i w1[i, b1] w2[i, b2];
  * loss L = mean_b (rho_b - target_b)^2.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import ndtr

from . import core, mmd


def frame(X0, V0, observer):
    """Orthonormal sky frame (e1, e2, n) of the present-day progenitor."""
    X0 = np.asarray(X0, float)
    V0 = np.asarray(V0, float)
    d = X0 - np.asarray(observer, float)
    e1 = d / np.linalg.norm(d)
    n = np.cross(d, V0)
    n /= np.linalg.norm(n)
    e2 = np.cross(n, e1)
    return e1, e2, n


def project(x, observer, fr):
    """(phi1, phi2) in radians of positions x (N, 3)."""
    e1, e2, n = fr
    d = np.asarray(x, float) - np.asarray(observer, float)
    p1, p2, p3 = d @ e1, d @ e2, d @ n
    r = np.sqrt(np.sum(d * d, axis=1))
    return np.arctan2(p2, p1), np.arcsin(p3 / r)


def project_vjp(x, observer, fr, g1, g2):
    """x-bar from phi1-bar (g1) and phi2-bar (g2)."""
    e1, e2, n = fr
    d = np.asarray(x, float) - np.asarray(observer, float)
    p1, p2, p3 = d @ e1, d @ e2, d @ n
    rho2 = np.sum(d * d, axis=1)
    q2 = p1 * p1 + p2 * p2
    # d phi1 / d d = (p1 e2 - p2 e1) / (p1^2 + p2^2)
    dphi1 = (p1[:, None] * e2[None, :] - p2[:, None] * e1[None, :]) / q2[:, None]
    # d phi2 / d d = (n |d|^2 - p3 d) / (|d|^2 sqrt(|d|^2 - p3^2))
    dphi2 = (n[None, :] * rho2[:, None] - p3[:, None] * d) / (
        rho2 * np.sqrt(rho2 - p3 * p3))[:, None]
    return g1[:, None] * dphi1 + g2[:, None] * dphi2


def edges(lo_deg, hi_deg, nb):
    return np.linspace(math.radians(lo_deg), math.radians(hi_deg), nb + 1)


def _weights(phi, e):
    """w[i, b] = Phi((e_{b+1} - phi_i)/s) - Phi((e_b - phi_i)/s), s = half a
    bin, and its derivative with respect to phi_i."""
    s = 0.5 * (e[1] - e[0])
    z = (e[None, :] - phi[:, None]) / s
    cdf = ndtr(z)
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    w = cdf[:, 1:] - cdf[:, :-1]
    dw = -(pdf[:, 1:] - pdf[:, :-1]) / s
    return w, dw


def soft_hist(phi1, phi2, e1, e2):
    w1, _ = _weights(phi1, e1)
    w2, _ = _weights(phi2, e2)
    return (w1.T @ w2) / phi1.shape[0]


def soft_hist_vjp(phi1, phi2, e1, e2, rho_bar):
    w1, dw1 = _weights(phi1, e1)
    w2, dw2 = _weights(phi2, e2)
    n = phi1.shape[0]
    g1 = np.sum(dw1 * (w2 @ rho_bar.T), axis=1) / n
    g2 = np.sum(dw2 * (w1 @ rho_bar), axis=1) / n
    return g1, g2


class StreamModel:
    """The mock-stream pipeline of Fig. 2 with a binned-density loss.

    cfg: a StreamC1-like config; xhat, vhat: the unit Plummer sample."""

    def __init__(self, cfg, xhat, vhat, n_steps=None):
        self.cfg = cfg
        self.xhat = np.asarray(xhat, float)
        self.vhat = np.asarray(vhat, float)
        self.N = self.xhat.shape[0]
        self.n_steps = cfg.n_steps if n_steps is None else n_steps
        self.fr = frame(cfg.X0, cfg.V0, cfg.observer)
        self.e1 = edges(*cfg.phi1_deg, cfg.nb1)
        self.e2 = edges(*cfg.phi2_deg, cfg.nb2)

    def physics(self, theta, pair):
        p = self.cfg.pot
        return core.Physics(G=self.cfg.G, eps=self.cfg.eps, pair=pair,
                            ext=core.NFW | core.MN, nfw_M=theta[2],
                            nfw_rs=p.nfw_rs, mn_M=theta[3], mn_a=p.mn_a,
                            mn_b=p.mn_b)

    def initial_state(self, theta):
        """Backward orbit of the centre of mass, then the shifted sphere."""
        t_acc, M_prog = theta[0], theta[1]
        n = self.n_steps
        Xi, Vi = core.integrate(self.physics(theta, False),
                                np.asarray(self.cfg.X0, float)[None, :],
                                np.asarray(self.cfg.V0, float)[None, :],
                                np.ones(1), -t_acc / n, n)
        a = self.cfg.a_prog
        x0 = a * self.xhat + Xi
        v0 = math.sqrt(self.cfg.G * M_prog / a) * self.vhat + Vi
        m = np.full(self.N, M_prog / self.N)
        return x0, v0, m

    def final_positions(self, theta):
        return self.final_state(theta)[0]

    def density(self, theta):
        xT = self.final_positions(theta)
        p1, p2 = project(xT, self.cfg.observer, self.fr)
        return soft_hist(p1, p2, self.e1, self.e2)

    def loss(self, theta, target):
        rho = self.density(theta)
        return float(np.mean((rho - target) ** 2))

    def loss_and_grad(self, theta, target):
        """Loss and dL/dTheta, Theta = (t_end, M_prog, M_NFW, M_MN)."""
        theta = [float(t) for t in theta]
        n = self.n_steps
        x0, v0, m = self.initial_state(theta)
        dt = theta[0] / n
        xT, _ = core.integrate(self.physics(theta, True), x0, v0, m, dt, n)
        p1, p2 = project(xT, self.cfg.observer, self.fr)
        rho = soft_hist(p1, p2, self.e1, self.e2)
        L = float(np.mean((rho - target) ** 2))
        rho_bar = 2.0 * (rho - target) / rho.size
        g1, g2 = soft_hist_vjp(p1, p2, self.e1, self.e2, rho_bar)
        xbar = project_vjp(xT, self.cfg.observer, self.fr, g1, g2)
        return L, self.theta_grad(theta, x0, v0, m, xbar, np.zeros_like(xbar))

    def final_state(self, theta):
        x0, v0, m = self.initial_state(theta)
        return core.integrate(self.physics(theta, True), x0, v0, m,
                              theta[0] / self.n_steps, self.n_steps)

    def mmd_loss(self, theta, Y, sigmas, mu=None, s=None):
        """MMD^2 between the simulated stream's phase-space cloud and the
        target cloud Y (m, 6) (the paper's point-cloud comparison)."""
        xT, vT = self.final_state([float(t) for t in theta])
        return float(mmd.mmd2(mmd.cloud(xT, vT), Y, sigmas, mu, s))

    def mmd_loss_and_grad(self, theta, Y, sigmas, mu=None, s=None):
        theta = [float(t) for t in theta]
        x0, v0, m = self.initial_state(theta)
        xT, vT = core.integrate(self.physics(theta, True), x0, v0, m,
                                theta[0] / self.n_steps, self.n_steps)
        L, g = mmd.mmd2_grad(mmd.cloud(xT, vT), Y, sigmas, mu, s)
        return float(L), self.theta_grad(theta, x0, v0, m, g[:, :3].copy(), g[:, 3:].copy())

    def theta_grad(self, theta, x0, v0, m, xbar, vbar):
        """dL/dTheta from dL/dx_T, dL/dv_T through the n-body run, the
        Plummer shift and the backward orbit."""
        t_acc, M_prog = theta[0], theta[1]
        n = self.n_steps
        a = self.cfg.a_prog
        G = self.cfg.G
        dt = t_acc / n
        r = core.vjp(self.physics(theta, True), x0, v0, m, dt, n, xbar, vbar)
        # initial-state adjoint: x0 = a xhat + X, v0 = sqrt(G M/a) vhat + V,
        # m_j = M / N
        Xb = r["x0bar"].sum(axis=0)
        Vb = r["v0bar"].sum(axis=0)
        Mb_v = 0.5 * math.sqrt(G / (a * M_prog)) * np.sum(r["v0bar"] * self.vhat)
        Mb_m = np.sum(r["mbar"]) / self.N
        Mb = Mb_v + Mb_m
        # backward orbit adjoint (single particle, external potential only)
        ro = core.vjp(self.physics(theta, False),
                      np.asarray(self.cfg.X0, float)[None, :],
                      np.asarray(self.cfg.V0, float)[None, :], np.ones(1),
                      -t_acc / n, n, Xb[None, :], Vb[None, :], want_mbar=False)
        # t_end enters twice, through the forward run's dt and the backward
        # orbit's -dt; the two parts are kept for error bounds
        self.t_end_parts = (r["dt_bar"] / n, -ro["dt_bar"] / n)
        # every component is a sum of two separately computed parts (the
        # n-body run's and the orbit's; for M_Plummer the velocity scaling's
        # and the masses'); kept for error bounds as well
        self.grad_parts = (np.array([r["dt_bar"] / n, Mb_v, r["nfw_M_bar"], r["mn_M_bar"]]),
                           np.array([-ro["dt_bar"] / n, Mb_m, ro["nfw_M_bar"],
                                     ro["mn_M_bar"]]))
        grad = np.array([
            r["dt_bar"] / n - ro["dt_bar"] / n,
            Mb,
            r["nfw_M_bar"] + ro["nfw_M_bar"],
            r["mn_M_bar"] + ro["mn_M_bar"],
        ])
        return grad

"""Orbit fitting of the progenitor and the Fisher matrix, FP64 numpy oracle.

TEST INFRASTRUCTURE ONLY.

The paper's second inference method (Sec. 2.2.2): a single particle, the
progenitor, is integrated forward and backward for up to 2 Gyr from its
present-day phase-space point in the external potential; its orbit is
projected onto the stream's frame (phi1, phi2, mu_phi1 cos phi2, mu_phi2,
v_h), interpolated along phi1 at the observed stream's phi1 values and
compared with them by a chi-square; the parameters are the NFW mass and
scale radius and the Miyamoto-Nagai mass, scale length and height; the
maximum-likelihood estimate comes from Levenberg-Marquardt and the Fisher
matrix is F = (1/2) d^2 chi^2 / d theta d theta.  Readings (the paper's
observations, frame, errors and window come from other work not in hand):

  * frame: e1 towards the present progenitor seen from the observer, pole
    n along (X0 - x_obs) x V0, e2 = n x e1 (the stream head's frame), so the
    progenitor sits at phi1 = phi2 = 0 and moves towards +phi1;
  * observer at x_obs with velocity v_obs; with d = x - x_obs, D = |d|,
    u = d / D, w = v - v_obs:
      phi1 = atan2(u.e2, u.e1), phi2 = asin(u.n),
      mu_phi1 cos phi2 = w.e_phi1 / D, mu_phi2 = w.e_phi2 / D (rad/Myr ->
      mas/yr by 206.264806...), v_h = w.u (kpc/Myr -> km/s),
      e_phi1 = -sin(phi1) e1 + cos(phi1) e2,
      e_phi2 = -sin(phi2) (cos(phi1) e1 + sin(phi1) e2) + cos(phi2) n;
  * the model arc: kick-drift-kick steps of dt from t = 0, forward while
    phi1 stays in the window and keeps increasing, backward (step -dt) while
    it stays in the window and keeps decreasing, each for at most t_max;
  * the model at an observed phi1: linear interpolation between the two arc
    points that bracket it; an observation beyond the arc's end takes the
    end point;
  * chi^2 = sum_obs sum_q (model_q - obs_q)^2 / sigma_q^2 over q = (phi2,
    mu_phi1 cos phi2, mu_phi2, v_h).

Everything here is the definition written out; derivatives are central
differences (Richardson) of chi^2, written in the tests.
"""
from __future__ import annotations

import numpy as np

from . import core
from .stream import frame

KMS = 1.0227121650537077e-3        # 1 km/s in kpc/Myr
MASYR = 206.26480624709636         # 1 rad/Myr in mas/yr


def observables(x, v, x_obs, v_obs, fr):
    """(phi1, phi2, mu_phi1 cos phi2 [mas/yr], mu_phi2 [mas/yr], v_h [km/s])
    of points x, v (k, 3)."""
    e1, e2, n = fr
    d = np.atleast_2d(x) - np.asarray(x_obs, float)
    w = np.atleast_2d(v) - np.asarray(v_obs, float)
    D = np.linalg.norm(d, axis=1)
    u = d / D[:, None]
    phi1 = np.arctan2(u @ e2, u @ e1)
    phi2 = np.arcsin(np.clip(u @ n, -1.0, 1.0))
    c1, s1 = np.cos(phi1), np.sin(phi1)
    c2, s2 = np.cos(phi2), np.sin(phi2)
    ep1 = -s1[:, None] * e1 + c1[:, None] * e2
    ep2 = -s2[:, None] * (c1[:, None] * e1 + s1[:, None] * e2) + c2[:, None] * n
    mu1 = np.sum(w * ep1, axis=1) / D * MASYR
    mu2 = np.sum(w * ep2, axis=1) / D * MASYR
    vh = np.sum(w * u, axis=1) / KMS
    return np.stack([phi1, phi2, mu1, mu2, vh], axis=1)


class OrbitFit:
    """chi^2 of the progenitor's orbit against an observed track."""

    def __init__(self, G, X0, V0, x_obs, v_obs, window, dt, t_max):
        self.G = G
        self.X0 = np.asarray(X0, float)
        self.V0 = np.asarray(V0, float)
        self.x_obs = np.asarray(x_obs, float)
        self.v_obs = np.asarray(v_obs, float)
        self.fr = frame(self.X0, self.V0, self.x_obs)
        self.window = (float(window[0]), float(window[1]))
        self.dt = float(dt)
        self.nmax = int(round(t_max / dt))

    def physics(self, theta):
        M_nfw, rs, M_mn, a, b = (float(t) for t in theta)
        return core.Physics(G=self.G, pair=False, ext=core.NFW | core.MN, nfw_M=M_nfw,
                            nfw_rs=rs, mn_M=M_mn, mn_a=a, mn_b=b)

    def half_arc(self, theta, sign):
        """Observables along one direction of the arc, starting at t = 0."""
        ph = self.physics(theta)
        x = self.X0[None, :].copy()
        v = self.V0[None, :].copy()
        pts = [observables(x, v, self.x_obs, self.v_obs, self.fr)[0]]
        lo, hi = self.window
        for _ in range(self.nmax):
            x, v = core.integrate(ph, x, v, np.ones(1), sign * self.dt, 1)
            q = observables(x, v, self.x_obs, self.v_obs, self.fr)[0]
            if not (lo <= q[0] <= hi) or sign * (q[0] - pts[-1][0]) <= 0.0:
                break
            pts.append(q)
        return np.array(pts)

    def arc(self, theta):
        """The arc through the progenitor, ordered by increasing phi1."""
        fwd = self.half_arc(theta, 1.0)
        bwd = self.half_arc(theta, -1.0)
        return np.concatenate([bwd[::-1], fwd[1:]])

    def model(self, theta, phi1_obs):
        """Model (phi2, mu1, mu2, v_h) at the observed phi1 values."""
        A = self.arc(theta)
        out = np.empty((len(phi1_obs), 4))
        for i, p in enumerate(phi1_obs):
            if p <= A[0, 0]:
                out[i] = A[0, 1:]
            elif p >= A[-1, 0]:
                out[i] = A[-1, 1:]
            else:
                k = int(np.searchsorted(A[:, 0], p)) - 1
                w = (p - A[k, 0]) / (A[k + 1, 0] - A[k, 0])
                out[i] = A[k, 1:] + w * (A[k + 1, 1:] - A[k, 1:])
        return out

    def chi2(self, theta, obs, sigma):
        """obs: (n_obs, 5) = phi1, phi2, mu1, mu2, v_h; sigma: 4 errors."""
        obs = np.asarray(obs, float)
        r = (self.model(theta, obs[:, 0]) - obs[:, 1:]) / np.asarray(sigma, float)[None, :]
        return float(np.sum(r * r))

    def residuals(self, theta, obs, sigma):
        obs = np.asarray(obs, float)
        return ((self.model(theta, obs[:, 0]) - obs[:, 1:]) /
                np.asarray(sigma, float)[None, :]).ravel()


def mock_observations(fit, theta, n_obs, phi1_range, sigma, seed):
    """An observed track: the model at theta at n_obs phi1 values spread
    uniformly over phi1_range, plus seeded Gaussian errors sigma."""
    phi1 = np.linspace(phi1_range[0], phi1_range[1], n_obs)
    clean = fit.model(theta, phi1)
    rng = np.random.default_rng(seed)
    noisy = clean + rng.normal(size=clean.shape) * np.asarray(sigma, float)[None, :]
    return np.concatenate([phi1[:, None], noisy], axis=1)


def fd_gradient(f, xi, h=1e-5):
    """Richardson central differences of f at xi."""
    g = np.zeros(len(xi))
    for k in range(len(xi)):
        e = np.zeros(len(xi))
        e[k] = h
        d1 = (f(xi + e) - f(xi - e)) / (2 * h)
        d2 = (f(xi + e / 2) - f(xi - e / 2)) / h
        g[k] = (4 * d2 - d1) / 3
    return g


def fd_hessian(f, xi, h=1e-3):
    """Second central differences of f at xi (symmetric)."""
    m = len(xi)
    H = np.zeros((m, m))
    f0 = f(xi)
    for a in range(m):
        ea = np.zeros(m)
        ea[a] = h
        H[a, a] = (f(xi + ea) - 2 * f0 + f(xi - ea)) / (h * h)
        for b in range(a + 1, m):
            eb = np.zeros(m)
            eb[b] = h
            H[a, b] = H[b, a] = (f(xi + ea + eb) - f(xi + ea - eb) - f(xi - ea + eb)
                                 + f(xi - ea - eb)) / (4 * h * h)
    return H

"""Orbit fitting and Fisher contours (the paper's second inference method,
Sec. 2.2.2) on a synthetic stream track.

  * observation: the progenitor's arc at theta_true = (M_NFW, r_s, M_MN,
    a_MN, b_MN) projected to (phi1, phi2, mu_phi1 cos phi2, mu_phi2, v_h),
    sampled at n_obs phi1 values, plus seeded Gaussian errors;
  * maximum-likelihood estimate: Levenberg-Marquardt from `starts` random
    points with 0.5 theta_true < theta < 2 theta_true (log-uniform), all
    starts at once (one GPU thread each), trial points kept within a decade
    of theta_true on either side; the lowest chi^2 wins;
  * Fisher matrix F = (1/2) d^2 chi^2 / d theta^2 at the estimate and at
    the truth (here in log10 theta, the paper's dex units) and the
    covariance C = F^-1.

The mock track is generated with the library's own arc (nbody_orbitfit_arc).

    python -m paper_2511_22468_gb300.orbitfit [--starts 1000] [--n-obs 64]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import nbody as nb
from .configs import C1, G_KPC_MSUN_MYR

KMS = 1.0227121650537077e-3
V_OBSERVER = np.array([12.9, 245.6, 7.78]) * KMS     # observer velocity, kpc/Myr
THETA_TRUE = np.array([1e12, 16.0, 6.8e10, 3.0, 0.28])
SIGMA = np.array([math.radians(0.1), 0.05, 0.05, 1.0])
NAMES = ("M_NFW", "r_s", "M_MN", "a_MN", "b_MN")


def config(window_deg=60.0, dt=0.5, t_max=2000.0, sigma=SIGMA):
    c = nb.nbody_orbitfit_cfg()
    c.G = G_KPC_MSUN_MYR
    c.X0[:] = list(C1.X0)
    c.V0[:] = list(C1.V0)
    c.observer[:] = list(C1.observer)
    c.observer_vel[:] = list(V_OBSERVER)
    c.phi1_lo, c.phi1_hi = math.radians(-window_deg), math.radians(window_deg)
    c.dt, c.t_max = dt, t_max
    c.sigma[:] = list(sigma)
    return c


def mock_track(n_obs=64, span_deg=40.0, seed=0, theta=THETA_TRUE, sigma=SIGMA):
    """Observed track: the arc at theta interpolated at n_obs phi1 values in
    [-span, span] degrees plus Gaussian errors sigma."""
    h = nb.nbody_orbitfit_create(config(), np.zeros((1, 5)))
    try:
        arc = nb.nbody_orbitfit_arc(h, theta)
    finally:
        nb.nbody_orbitfit_destroy(h)
    phi1 = np.linspace(math.radians(-span_deg), math.radians(span_deg), n_obs)
    clean = np.stack([np.interp(phi1, arc[:, 0], arc[:, k]) for k in range(1, 5)], axis=1)
    rng = np.random.default_rng(seed)
    return np.concatenate([phi1[:, None], clean + rng.normal(size=clean.shape) * sigma], axis=1)


def fisher_summary(h, theta):
    """Fisher matrix F = (1/2) d^2 chi^2 in dex at theta (exact, second-order
    duals) and its covariance F^-1; where F is not positive definite (a
    point that is not a minimum) the Gauss-Newton matrix, positive
    semi-definite by construction, gives the covariance instead."""
    F_ln, Fgn_ln = nb.nbody_orbitfit_fisher(h, theta)
    s = math.log(10.0) ** 2                 # d/d log10 theta = ln 10 d/d ln theta
    F_dex, Fgn_dex = F_ln * s, Fgn_ln * s
    eig = np.linalg.eigvalsh(F_dex)
    use = F_dex if eig.min() > 0 else Fgn_dex
    cov = np.linalg.pinv(use)
    sig = np.sqrt(np.maximum(np.diag(cov), 0.0))
    return {"sigma_dex": dict(zip(NAMES, sig.tolist())),
            "covariance_from": "hessian" if eig.min() > 0 else "gauss_newton",
            "correlation": np.round(cov / np.outer(sig, sig), 4).tolist(),
            "eig_hessian": eig.tolist(),
            "eig_gauss_newton": np.linalg.eigvalsh(Fgn_dex).tolist(),
            "gauss_newton_vs_hessian_max_rel":
                float(np.max(np.abs(Fgn_ln - F_ln)) / np.max(np.abs(F_ln)))}, sig


def run(starts=1000, n_obs=64, seed=0, max_iter=200):
    obs = mock_track(n_obs=n_obs, seed=seed)
    h = nb.nbody_orbitfit_create(config(), obs)
    rng = np.random.default_rng(seed + 1)
    th0 = THETA_TRUE[None, :] * np.exp(rng.uniform(math.log(0.5), math.log(2.0), (starts, 5)))
    t0 = time.perf_counter()
    th, chi2, its = nb.nbody_orbitfit_lm(h, th0, max_iter=max_iter, lo=THETA_TRUE / 10,
                                         hi=THETA_TRUE * 10)
    t_lm = time.perf_counter() - t0
    k = int(np.argmin(chi2))
    best = th[k]
    t0 = time.perf_counter()
    at_mle, sig = fisher_summary(h, best)
    t_f = time.perf_counter() - t0
    at_truth, _ = fisher_summary(h, THETA_TRUE)
    nb.nbody_orbitfit_destroy(h)
    err_dex = np.log10(best / THETA_TRUE)
    near = np.mean(chi2 <= chi2[k] + 1.0)
    at_mle.update({"error_dex": dict(zip(NAMES, err_dex.tolist())),
                   "pull": dict(zip(NAMES, (err_dex / sig).tolist()))})
    return {"workload": {"starts": starts, "n_obs": n_obs, "residuals": 4 * n_obs,
                         "theta_true": THETA_TRUE.tolist(), "sigma": SIGMA.tolist(),
                         "window_deg": 60.0, "dt_myr": 0.5, "t_max_myr": 2000.0},
            "lm": {"time_s": t_lm, "starts_per_s": starts / t_lm,
                   "median_iterations": float(np.median(its)),
                   "converged_fraction": float(np.mean(its < max_iter)),
                   "best_chi2": float(chi2[k]), "fraction_within_1_of_best": float(near),
                   "best_theta": best.tolist()},
            "fisher_at_mle": at_mle, "fisher_time_s": t_f, "fisher_at_truth": at_truth}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--starts", type=int, default=1000)
    ap.add_argument("--n-obs", type=int, default=64)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    from . import build
    build.build()
    print(json.dumps(run(starts=a.starts, n_obs=a.n_obs, seed=a.seed)))


if __name__ == "__main__":
    main()

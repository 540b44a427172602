"""Parameter recovery to a fixed parameter error: the plain method, the
batched form and the learned warm start (the stream workload; Sec. 2.2.1,
Fig. 2; the neural-network coupling of Sec. 3).

Experiment (stream workload, N = 1e4, at a horizon where the discrete adjoint
is a descent direction: 100 Myr; at 200 Myr it points away from the truth
at some prior points, and the full 3 Gyr gradient is dominated by the
chaotic growth of the progenitor's adjoint):

  * observation: the simulated stream at theta_obs = theta_c * f_obs, a point
    inside the +-30 % prior around the centre theta_c, from the same unit
    Plummer sample as every simulation (common random numbers);
  * loss: the paper's point-cloud comparison, MMD^2 of the final 6-D
    phase-space cloud against the observed one (bandwidths 0.5, 1, 2 in the
    observation's standard deviations);
  * target: max_k |theta_k / theta_obs_k - 1| <= err_target (5 %), measured
    at the minimum-loss estimate (Fig. 2 step 5);
  * plain: gradient descent (Adam on normalised parameters, simulator
    adjoint gradient, a step that raises the loss is undone and the rate
    halved) from theta_c, one simulation per launch with the launch shapes
    tuned for its size; a descent from a warm
    start (the batched grid's best point, the surrogate's inversion) starts
    with a quarter of the rate, its start being several times closer;
  * batched: the paper's grid stage on the batched kernel -- every call one
    persistent launch per step for all 81 points of a 3^4 pattern around the
    current estimate, the pattern halved when its centre is best -- then the
    same adjoint descent from the best point;
  * surrogate: binned sky densities (a 32 x 32 window scaled to the stream's
    extent at this horizon) of n_train prior samples from the batched kernel,
    the network trained on them by the library's kernels and inverted for the
    observed density, then the plain descent from there.  Its time is given
    with and without the one-off data generation and training;
  * surrogate + grid: the same inversion as the start of the batched grid
    stage, whose first spacing per parameter is twice the surrogate's rms
    inversion error on validation densities (measured once after training:
    the spread the surrogate leaves in each parameter), then the descent.
Every final parameter comes from the simulator-gradient descent.

    python -m paper_2511_22468_gb300.warmstart [--n 10000] [--t-end 100]
        [--err-target 0.05] [--n-train 3584] [--epochs 300] [--n-random K]
"""
from __future__ import annotations

import argparse
import dataclasses
import itertools
import json
import time

import numpy as np
import torch

from .configs import C1, C4
from .inputs import plummer_unit, uniform_factors
from .stream import StreamBatch, StreamModel
from .surrogate import DENSITY_SCALE, EnsembleDensities, Surrogate, descend, from_u

F_OBS = (1.15, 0.85, 1.2, 0.8)
# observations (factors of the prior centre) of the recovery experiment
F_OBS_LIST = ((1.15, 0.85, 1.2, 0.8), (0.9, 1.2, 0.85, 1.15), (1.2, 1.1, 0.9, 0.75))
SIGMAS = (0.5, 1.0, 2.0)


def pattern_search(batch, centre, width, theta_true, err_target, s0=0.5, s_min=0.02,
                   max_calls=30, clock=time.perf_counter, u_start=None):
    """The grid stage on the batched pipeline: each call evaluates the loss
    at the 81 points c + s * {-1, 0, 1}^4 (normalised parameters, c = 0, the
    prior centre, unless u_start is given; s a number or one spacing per
    parameter) as members of one batch; the best point becomes the new c,
    and the spacing halves when c itself is best.
    Returns the trajectory of estimates (the best point so far after every
    call)."""
    centre = np.asarray(centre, float)
    grid = np.array(list(itertools.product((-1.0, 0.0, 1.0), repeat=4)))
    t0 = clock()
    c = np.zeros(4) if u_start is None else np.clip(np.asarray(u_start, float), -1.5, 1.5)
    s = np.asarray(s0, float) * np.ones(4)  # spacing per parameter
    best_L, best_u = np.inf, c.copy()
    traj = []
    for call in range(max_calls):
        U = np.clip(c[None, :] + s * grid, -1.5, 1.5)
        L = batch.loss(from_u(U, centre, width))
        k = int(np.argmin(L))
        if L[k] < best_L:
            best_L, best_u = float(L[k]), U[k].copy()
        if np.array_equal(U[k], c) or not L[k] < np.inf:
            s *= 0.5
        c = best_u.copy()
        th = from_u(best_u, centre, width)
        err = float(np.max(np.abs(th / theta_true - 1.0)))
        traj.append({"iter": call, "t": clock() - t0, "loss": best_L, "err": err,
                     "theta": th.tolist(), "spacing": s.tolist()})
        if err <= err_target or np.max(s) < s_min:
            break
    return traj


def time_to_err(tr, err_target):
    for row in tr:
        if row["err"] is not None and row["err"] <= err_target:
            return row["t"]
    return None


def summary(tr, err_target, t_pre=0.0, extra=None):
    t_hit = time_to_err(tr, err_target)
    s = {"iters": len(tr) - 1, "reached": t_hit is not None,
         "time_to_target_s": None if t_hit is None else t_hit + t_pre, "pre_s": t_pre,
         "start_err": tr[0]["err"], "final_err": tr[-1]["err"], "final_loss": tr[-1]["loss"],
         "final_theta": tr[-1]["theta"], "err_trace": [r["err"] for r in tr]}
    if extra:
        s.update(extra)
    return s


def run(n=10_000, t_end=100.0, err_target=0.05, n_train=3584, n_val=512, epochs=300,
        max_iters=200, lr=0.2, lr_warm=0.05, window=(1.0, 0.5), observations=F_OBS_LIST,
        grid_s0=0.37, n_calib=16, device="cuda:0", n_random=0, random_seed=777):
    dev = torch.device(device)
    steps = int(round(t_end / 0.5))
    cfg = dataclasses.replace(C1, n=n, t_acc=float(t_end), n_steps=steps,
                              phi1_deg=(-window[0], window[0]), phi2_deg=(-window[1], window[1]))
    xh, vh = plummer_unit(n, cfg.seed)
    centre = np.array(cfg.theta_true, float)
    width = C4.width
    sync = lambda: torch.cuda.synchronize(dev)  # noqa: E731
    out = {"workload": {"n": n, "t_end_myr": t_end, "steps": steps,
                        "theta_centre": centre.tolist(), "prior_width": width,
                        "loss": "MMD^2 of the 6-D cloud, sigma 0.5/1/2",
                        "err_target": err_target, "density_window_deg": list(window),
                        "descent_lr": lr, "descent_lr_warm": lr_warm,
                        "grid_spacing0": grid_s0}}

    # the surrogate, once: training densities from the batched kernel, training
    f = uniform_factors(n_train + n_val, width, 4, C4.seed_params)
    gen = EnsembleDensities(cfg, xh, vh, device=device)
    sync()
    t0 = time.perf_counter()
    Y = gen.densities(centre * f) * DENSITY_SCALE
    t_gen = time.perf_counter() - t0
    gen.close()
    U = (f - 1.0) / width
    net = Surrogate(device=device)
    sync()
    t0 = time.perf_counter()
    hist = net.fit(U[:n_train], Y[:n_train], epochs=epochs, lr=1e-3, batch=256,
                   U_val=U[n_train:], Y_val=Y[n_train:], log_every=max(1, epochs // 10))
    sync()
    t_train = time.perf_counter() - t0
    # the surrogate's spread per parameter: rms inversion error (normalised
    # units) on n_calib validation densities; the warm grid stage's spacing
    t0 = time.perf_counter()
    u_cal = np.array([net.invert(Y[n_train + i])[0] for i in range(n_calib)])
    sigma_u = np.sqrt(np.mean((u_cal - U[n_train:n_train + n_calib]) ** 2, axis=0))
    t_cal = time.perf_counter() - t0
    s0_warm = np.clip(2.0 * sigma_u, 0.1, 0.6)
    t_train += t_cal
    out["surrogate_training"] = {"data_generation_s": t_gen, "n_train": n_train,
                                 "n_val": n_val, "training_s": t_train,
                                 "calibration_s": t_cal, "inversion_rms_u": sigma_u.tolist(),
                                 "grid_spacing0_warm": s0_warm.tolist(),
                                 "val_mse": hist[-1].get("val_mse")}
    if n_random:
        observations = tuple(observations) + tuple(
            tuple(float(v) for v in f) for f in
            uniform_factors(n_random, 0.8 * width, 4, random_seed))

    model = StreamModel(cfg, xh, vh, device=device)
    # the single-system pipeline takes the launch shapes tuned for this size,
    # as the batched stage does (one-off, not timed)
    model.autotune(list(centre))
    runs = []
    for fo in observations:
        theta_obs = centre * np.array(fo)
        xt, vt = model.final_state(list(theta_obs))
        rho_obs = model.density(list(theta_obs)).cpu().numpy().ravel()
        model.set_target_cloud(xt, vt, SIGMAS)
        L_c = model.loss_and_grad(list(centre))[0]  # also the first (warm-up) gradient
        r = {"f_obs": list(fo), "theta_obs": theta_obs.tolist(), "loss_centre": L_c,
             "err_centre": float(np.max(np.abs(centre / theta_obs - 1.0)))}

        # plain: descent from the prior centre, one simulation per launch
        sync()
        tr = descend(model, centre, centre, width, lr=lr, max_iters=max_iters,
                     theta_true=theta_obs, err_target=err_target)
        r["plain"] = summary(tr, err_target, extra={"gradients": len(tr)})

        # batched: the grid stage (81 members per call), then the descent
        X = xt.detach().cpu().numpy().T
        Vv = vt.detach().cpu().numpy().T
        sb = StreamBatch(cfg, xh, vh, np.stack([X] * 81), np.stack([Vv] * 81), SIGMAS)
        sb.loss(np.repeat(centre[None, :], 81, axis=0))  # first call: launch-shape tuning
        sync()
        t0 = time.perf_counter()
        grid = pattern_search(sb, centre, width, theta_obs, err_target, s0=grid_s0)
        t_grid = time.perf_counter() - t0
        tr = descend(model, np.array(grid[-1]["theta"]), centre, width, lr=lr_warm,
                     max_iters=max_iters, theta_true=theta_obs, err_target=err_target)
        r["batched"] = summary(tr, err_target, t_pre=t_grid,
                               extra={"grid_calls": len(grid), "members_per_call": 81,
                                      "grid_s": t_grid, "grid_err": grid[-1]["err"],
                                      "gradients": len(tr)})

        # surrogate: inversion of the observed density, then the descent
        t0 = time.perf_counter()
        u0, inv_loss = net.invert(rho_obs * DENSITY_SCALE)
        theta0 = from_u(u0, centre, width)
        t_inv = time.perf_counter() - t0
        tr = descend(model, theta0, centre, width, lr=lr_warm, max_iters=max_iters,
                     theta_true=theta_obs, err_target=err_target)
        t_hit = time_to_err(tr, err_target)
        r["surrogate"] = summary(
            tr, err_target, t_pre=t_inv,
            extra={"gradients": len(tr), "inversion_s": t_inv, "theta0": theta0.tolist(),
                   "theta0_err": float(np.max(np.abs(theta0 / theta_obs - 1))),
                   "inversion_loss": inv_loss,
                   "time_incl_data_and_training_s":
                       None if t_hit is None else t_hit + t_inv + t_gen + t_train})

        # surrogate + grid: the grid stage started at the inverted point with
        # the smaller spacing, then the descent from its best point
        sync()
        t0 = time.perf_counter()
        u0, _ = net.invert(rho_obs * DENSITY_SCALE)
        grid = pattern_search(sb, centre, width, theta_obs, err_target, s0=s0_warm,
                              u_start=u0)
        t_pre = time.perf_counter() - t0
        tr = descend(model, np.array(grid[-1]["theta"]), centre, width, lr=lr_warm,
                     max_iters=max_iters, theta_true=theta_obs, err_target=err_target)
        t_hit = time_to_err(tr, err_target)
        r["surrogate_grid"] = summary(
            tr, err_target, t_pre=t_pre,
            extra={"grid_calls": len(grid), "members_per_call": 81,
                   "inversion_and_grid_s": t_pre, "grid_err": grid[-1]["err"],
                   "gradients": len(tr),
                   "time_incl_data_and_training_s":
                       None if t_hit is None else t_hit + t_pre + t_gen + t_train})
        sb.close()
        runs.append(r)
    out["observations"] = runs
    for k in ("plain", "batched", "surrogate", "surrogate_grid"):
        ts = [r[k]["time_to_target_s"] for r in runs]
        out[k + "_reached"] = sum(t is not None for t in ts)
        out[k + "_median_time_to_target_s"] = (float(np.median([t for t in ts if t is not None]))
                                             if any(t is not None for t in ts) else None)
    net.close()
    model.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=10_000)
    ap.add_argument("--t-end", type=float, default=100.0)
    ap.add_argument("--err-target", type=float, default=0.05)
    ap.add_argument("--n-train", type=int, default=3584)
    ap.add_argument("--n-val", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--max-iters", type=int, default=200)
    ap.add_argument("--lr", type=float, default=0.2)
    ap.add_argument("--n-random", type=int, default=0,
                    help="observations drawn from the inner 80 %% of the prior, besides the three "
                         "fixed ones")
    a = ap.parse_args()
    from . import build
    build.build()
    res = run(n=a.n, t_end=a.t_end, err_target=a.err_target, n_train=a.n_train,
              n_val=a.n_val, epochs=a.epochs, max_iters=a.max_iters, lr=a.lr,
              n_random=a.n_random)
    print(json.dumps(res))


if __name__ == "__main__":
    main()

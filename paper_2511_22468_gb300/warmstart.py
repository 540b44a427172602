"""Parameter recovery with and without the learned warm start.

Experiment (stream workload at a horizon where the discrete adjoint is
informative; the horizon sweep of stream.py shows the full 3 Gyr gradient is
dominated by the chaotic growth of the progenitor's adjoint):

  * observation: the simulated density at theta_obs = theta_c * f_obs, a
    point inside the +-30 % prior around the centre theta_c;
  * target: a recovery loss tau = tau_frac * L(theta_c);
  * plain: gradient descent (Adam on normalised parameters, simulator
    adjoint gradient) from theta_c, one simulation per launch;
  * batched: one 64-member batch of prior samples (one persistent pair
    launch per step for all members) -> best member -> the same descent;
  * surrogate: densities of n_train prior samples from the batched kernel,
    the network trained on them, inverted for the observation -> the same
    descent.  Times are reported with and without the one-off data
    generation and training.
Every final parameter comes from the simulator-gradient descent.

    python -m paper_2511_22468_gb300.warmstart [--n 10000] [--t-end 200]
        [--n-train 3584] [--n-val 512] [--epochs 300] [--max-iters 40]
        [--tau-frac 0.02]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import time

import numpy as np
import torch

from .configs import C1, C4
from .inputs import plummer_unit, uniform_factors
from .stream import StreamModel
from .surrogate import DENSITY_SCALE, EnsembleDensities, Surrogate, descend, from_u, to_u

F_OBS = (1.15, 0.85, 1.2, 0.8)


def run(n=10_000, t_end=200.0, n_train=3584, n_val=512, epochs=300, max_iters=40,
        tau_frac=2e-2, lr=0.05, seed=0, device="cuda:0"):
    dev = torch.device(device)
    steps = int(round(t_end / 0.5))
    cfg = dataclasses.replace(C1, n=n, t_acc=float(t_end), n_steps=steps)
    xh, vh = plummer_unit(n, cfg.seed)
    centre = np.array(cfg.theta_true, float)
    width = C4.width
    theta_obs = centre * np.array(F_OBS)
    sync = lambda: torch.cuda.synchronize(dev)  # noqa: E731

    model = StreamModel(cfg, xh, vh, device=device)
    target = model.density(theta_obs)
    model.set_target(target)
    L_c = model.loss(centre)
    tau = tau_frac * L_c
    out = {"workload": {"n": n, "t_end_myr": t_end, "steps": steps, "theta_centre": centre.tolist(),
                        "theta_obs": theta_obs.tolist(), "prior_width": width,
                        "loss_centre": L_c, "tau": tau}}

    # plain: descent from the prior centre
    sync()
    tr = descend(model, centre, centre, width, lr=lr, max_iters=max_iters, loss_target=tau,
                 theta_true=theta_obs)
    out["plain"] = summary(tr, tau)

    # batched: one batch of prior samples, best member, then descent
    rng_f = uniform_factors(64, width, 4, seed + 7)
    gen = EnsembleDensities(cfg, xh, vh, batch=64, device=device)
    sync()
    t0 = time.perf_counter()
    thetas = centre * rng_f
    rho = gen.densities(thetas)
    Ls = np.mean((rho - target.cpu().numpy().reshape(1, -1)) ** 2, axis=1)
    best = thetas[int(np.argmin(Ls))]
    t_search = time.perf_counter() - t0
    tr = descend(model, best, centre, width, lr=lr, max_iters=max_iters, loss_target=tau,
                 theta_true=theta_obs)
    out["batched"] = summary(tr, tau, t_pre=t_search, extra={"best_sample_loss": float(Ls.min())})

    # surrogate: training data from the batched kernel, training, inversion
    f = uniform_factors(n_train + n_val, width, 4, C4.seed_params)
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
    t0 = time.perf_counter()
    u0, inv_loss = net.invert(target.cpu().numpy() * DENSITY_SCALE)
    theta0 = from_u(u0, centre, width)
    t_inv = time.perf_counter() - t0
    tr = descend(model, theta0, centre, width, lr=lr, max_iters=max_iters, loss_target=tau,
                 theta_true=theta_obs)
    out["surrogate"] = summary(tr, tau, t_pre=t_inv,
                               extra={"data_generation_s": t_gen, "n_train": n_train,
                                      "n_val": n_val, "training_s": t_train,
                                      "inversion_s": t_inv, "theta0": theta0.tolist(),
                                      "theta0_err": float(np.max(np.abs(theta0 / theta_obs - 1))),
                                      "inversion_loss": inv_loss, "history": hist,
                                      "time_incl_data_and_training_s":
                                          None if out_time(tr, tau) is None else
                                          out_time(tr, tau) + t_inv + t_gen + t_train})
    net.close()
    model.close()
    return out


def out_time(tr, tau):
    for row in tr:
        if row["loss"] <= tau:
            return row["t"]
    return None


def summary(tr, tau, t_pre=0.0, extra=None):
    t_hit = out_time(tr, tau)
    s = {"iters": len(tr) - 1, "reached": t_hit is not None,
         "time_to_target_s": None if t_hit is None else t_hit + t_pre,
         "pre_s": t_pre, "final_loss": tr[-1]["loss"], "final_err": tr[-1]["err"],
         "start_loss": tr[0]["loss"], "start_err": tr[0]["err"],
         "final_theta": tr[-1]["theta"],
         "loss_trace": [r["loss"] for r in tr]}
    if extra:
        s.update(extra)
    return s


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=10_000)
    ap.add_argument("--t-end", type=float, default=200.0)
    ap.add_argument("--n-train", type=int, default=3584)
    ap.add_argument("--n-val", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--max-iters", type=int, default=40)
    ap.add_argument("--tau-frac", type=float, default=2e-2)
    a = ap.parse_args()
    from . import build
    build.build()
    res = run(n=a.n, t_end=a.t_end, n_train=a.n_train, n_val=a.n_val, epochs=a.epochs,
              max_iters=a.max_iters, tau_frac=a.tau_frac)
    print(json.dumps(res))


if __name__ == "__main__":
    main()

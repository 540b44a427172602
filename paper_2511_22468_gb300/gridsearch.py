"""Grid search and gradient refinement with the point-cloud loss (the
paper's first inference method, Sec. 2.2.1 and Fig. 2).

  * observation: the simulated stream (final phase-space cloud) at theta_obs;
  * grid: a regular grid of per_dim^4 parameter vectors theta = (t_end,
    M_Plummer, M_NFW, M_MN) over the box theta_c (1 +- width), cell centres;
  * every grid point is simulated -- backward orbit of the centre of mass,
    Plummer sphere, forward n-body run -- as members of one batch context
    (one persistent pair launch per step for all members, graph-captured)
    and scored by MMD^2 against the observation (one batched MMD launch);
  * refinement: gradient descent from the best grid point with the
    pipeline's discrete-adjoint gradient of the same MMD^2 (the paper runs
    10 such steps); the estimate is the minimum-loss iterate.

The paper's workload is 10^4 grid points of 1000 particles and 1000 steps;
the default here keeps the stream workload's step (0.5 Myr), so 1000 steps
cover t_end = 500 Myr.

    python -m paper_2511_22468_gb300.gridsearch [--n 1000] [--steps 1000]
        [--per-dim 10] [--batch 1024] [--refine 10]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import time

import numpy as np
import torch

from . import nbody as nb
from .configs import C1
from .inputs import plummer_unit
from .stream import StreamModel


def regular_grid(centre, width, per_dim):
    """Cell centres of a per_dim^4 grid over centre * (1 +- width)."""
    f = 1.0 - width + (2.0 * width) * (np.arange(per_dim) + 0.5) / per_dim
    g = np.stack(np.meshgrid(f, f, f, f, indexing="ij"), axis=-1).reshape(-1, 4)
    return np.asarray(centre, float)[None, :] * g


class GridSearch:
    """MMD^2 of many parameter vectors against one observed cloud."""

    def __init__(self, cfg, xhat, vhat, tx, tv, sigmas=(0.5, 1.0, 2.0), batch=1024,
                 device="cuda:0", tuning=None):
        self.dev = torch.device(device)
        self.cfg = cfg
        self.model = StreamModel(cfg, xhat, vhat, device=device)
        self.n = n = self.model.n
        self.B = B = batch
        self.steps = cfg.n_steps
        offs = np.arange(B + 1) * n
        self.h = nb.nbody_create_batch(offs, [self._params(cfg.theta_true, (0,) * 6)] * B)
        self.tuning = tuning
        self.mmd = nb.nbody_mmd_create(n, B, torch.as_tensor(tx).to(self.dev).contiguous(),
                                       torch.as_tensor(tv).to(self.dev).contiguous(),
                                       list(sigmas))
        self.X = torch.empty((3, B * n), dtype=torch.float64, device=self.dev)
        self.V = torch.empty_like(self.X)
        self.M = torch.empty(B * n, dtype=torch.float64, device=self.dev)
        self.XO = torch.empty_like(self.X)
        self.VO = torch.empty_like(self.X)
        self.com = np.zeros((B, 6))
        self.L = torch.empty(B, dtype=torch.float64, device=self.dev)
        self.times = {"initial_states_s": 0.0, "simulate_s": 0.0, "mmd_s": 0.0}

    def _params(self, th, com):
        c, p = self.cfg, self.cfg.pot
        return nb.make_params(c.G, c.eps, th[0] / c.n_steps, ext_flags=3, nfw_M=th[2],
                              nfw_rs=p.nfw_rs, mn_M=th[3], mn_a=p.mn_a, mn_b=p.mn_b,
                              center=com[:3], center_vel=com[3:6],
                              center_mode=nb.NBODY_CENTER_GUIDE)

    def losses(self, thetas):
        thetas = np.asarray(thetas, float).reshape(-1, 4)
        out = np.empty(len(thetas))
        B = self.B
        sync = lambda: torch.cuda.synchronize(self.dev)  # noqa: E731
        for c0 in range(0, len(thetas), B):
            chunk = thetas[c0:c0 + B]
            full = np.concatenate([chunk, np.repeat(chunk[-1:], B - len(chunk), axis=0)])
            sync()
            t0 = time.perf_counter()
            nb.nbody_stream_initial_states(self.model.h, full, self.X, self.V, self.M, self.com)
            nb.nbody_set_params_batch(self.h, [self._params(th, cm)
                                               for th, cm in zip(full, self.com)])
            nb.nbody_set_state(self.h, self.X, self.V, self.M)
            if self.tuning is None:
                from . import autotune
                self.tuning, _, _ = autotune.tune(self.h, [self.n] * B,
                                                  torch.cuda.get_device_name(self.dev),
                                                  probe_steps=2)
            nb.nbody_set_tuning(self.h, self.tuning)
            sync()
            t1 = time.perf_counter()
            nb.nbody_integrate(self.h, self.steps)
            nb.nbody_get_state(self.h, self.XO, self.VO)
            sync()
            t2 = time.perf_counter()
            nb.nbody_mmd_eval_batch(self.mmd, B, self.XO, self.VO, self.L)
            out[c0:c0 + len(chunk)] = self.L.cpu().numpy()[:len(chunk)]
            t3 = time.perf_counter()
            self.times["initial_states_s"] += t1 - t0
            self.times["simulate_s"] += t2 - t1
            self.times["mmd_s"] += t3 - t2
        return out

    def close(self):
        if self.h is not None:
            nb.nbody_destroy(self.h)
            self.h = None
        if self.mmd is not None:
            nb.nbody_mmd_destroy(self.mmd)
            self.mmd = None
        self.model.close()


def refine(model, theta0, centre, width, iters=10, lr=0.05):
    """Adam in normalised parameters with the discrete-adjoint gradient;
    returns the trajectory (the minimum-loss iterate is the estimate)."""
    from .surrogate import descend
    return descend(model, theta0, centre, width, lr=lr, max_iters=iters)


def run(n=1000, steps=1000, t_end=500.0, per_dim=10, batch=1024, refine_iters=10,
        sigmas=(0.5, 1.0, 2.0), f_obs=(1.1, 0.9, 1.15, 0.85), width=0.3, seed=1,
        device="cuda:0", tuning=None):
    cfg = dataclasses.replace(C1, n=n, n_steps=steps, t_acc=float(t_end))
    centre = np.array(cfg.theta_true, float)
    theta_obs = centre * np.array(f_obs)
    xh, vh = plummer_unit(n, seed)
    obs = StreamModel(cfg, xh, vh, device=device)
    tx, tv = obs.final_state(list(theta_obs))
    obs.close()
    gs = GridSearch(cfg, xh, vh, tx, tv, sigmas=sigmas, batch=batch, device=device,
                    tuning=tuning)
    grid = regular_grid(centre, width, per_dim)
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    L = gs.losses(grid)
    t_grid = time.perf_counter() - t0
    k = int(np.argmin(L))
    best = grid[k]
    inter = float(n) ** 2 * steps * len(grid)
    res = {"workload": {"n": n, "steps": steps, "t_end_myr": t_end, "grid_points": len(grid),
                        "per_dim": per_dim, "batch": batch, "sigmas": list(sigmas),
                        "theta_obs": theta_obs.tolist(), "prior_width": width},
           "grid": {"time_s": t_grid, "sims_per_s": len(grid) / t_grid,
                    "pair_interactions_per_s": inter / gs.times["simulate_s"],
                    "breakdown_s": dict(gs.times), "launch_shape": gs.tuning,
                    "best_theta": best.tolist(),
                    "best_loss": float(L[k]),
                    "best_err": float(np.max(np.abs(best / theta_obs - 1)))}}
    gs.close()
    if refine_iters > 0:
        model = StreamModel(cfg, xh, vh, device=device)
        model.set_target_cloud(tx, tv, sigmas)
        t0 = time.perf_counter()
        tr = refine(model, best, centre, width, iters=refine_iters)
        t_ref = time.perf_counter() - t0
        res["refine"] = {"iters": len(tr) - 1, "time_s": t_ref, "final_theta": tr[-1]["theta"],
                         "final_loss": tr[-1]["loss"],
                         "final_err": float(np.max(np.abs(np.array(tr[-1]["theta"]) /
                                                          theta_obs - 1))),
                         "loss_trace": [r["loss"] for r in tr]}
        model.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1000)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--t-end", type=float, default=500.0)
    ap.add_argument("--per-dim", type=int, default=10)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--refine", type=int, default=10)
    a = ap.parse_args()
    from . import build
    build.build()
    print(json.dumps(run(n=a.n, steps=a.steps, t_end=a.t_end, per_dim=a.per_dim,
                         batch=a.batch, refine_iters=a.refine)))


if __name__ == "__main__":
    main()

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
    10 such steps); the estimate is the minimum-loss iterate;
  * bootstrap (--bootstrap R): the observation is redrawn R times from its
    observational errors (Gaussian per coordinate: --sigma-x kpc and
    --sigma-v km/s, or by default 5 % of the observed cloud's spread in
    that coordinate) and the grid stage is repeated for every
    realisation.  The grid's simulated clouds do not depend on the
    observation, so they are simulated once and kept in device memory
    (48 B per particle, 480 MB for 10^4 clouds of 1000); one call then
    scores every cloud against every realisation (nbody_mmd_eval_cross),
    and the spread of the per-realisation best grid points is the
    bootstrap distribution.  --bootstrap-refine K adds the gradient
    refinement for the first K realisations, many at once (one batched
    pipeline whose members each compare with their own realisation).

The paper's workload is 10^4 grid points of 1000 particles and 1000 steps;
the default here keeps the stream workload's step (0.5 Myr), so 1000 steps
cover t_end = 500 Myr.

    python -m paper_2511_22468_gb300.gridsearch [--n 1000] [--steps 1000]
        [--per-dim 10] [--batch 1024] [--refine 10] [--bootstrap R]
        [--bootstrap-refine K]
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
from .inputs import perturbed_clouds, plummer_unit
from .stream import StreamBatch, StreamModel
from .surrogate import descend_batch


def regular_grid(centre, width, per_dim):
    """Cell centres of a per_dim^4 grid over centre * (1 +- width)."""
    f = 1.0 - width + (2.0 * width) * (np.arange(per_dim) + 0.5) / per_dim
    g = np.stack(np.meshgrid(f, f, f, f, indexing="ij"), axis=-1).reshape(-1, 4)
    return np.asarray(centre, float)[None, :] * g


class GridSearch:
    """MMD^2 of many parameter vectors against one observed cloud."""

    def __init__(self, cfg, xhat, vhat, tx, tv, sigmas=(0.5, 1.0, 2.0), batch=1024,
                 device="cuda:0", tuning=None, keep_clouds=0):
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
        # every simulated cloud, kept for scoring against other observations
        self.CX = self.CV = None
        if keep_clouds:
            self.CX = torch.empty((3, keep_clouds * n), dtype=torch.float64, device=self.dev)
            self.CV = torch.empty_like(self.CX)

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
            if self.CX is not None:
                k = len(chunk) * self.n
                self.CX[:, c0 * self.n:c0 * self.n + k] = self.XO[:, :k]
                self.CV[:, c0 * self.n:c0 * self.n + k] = self.VO[:, :k]
            t3 = time.perf_counter()
            self.times["initial_states_s"] += t1 - t0
            self.times["simulate_s"] += t2 - t1
            self.times["mmd_s"] += t3 - t2
        return out

    def cross_losses(self, count, tx, tv):
        """MMD^2 of the first `count` kept clouds against each of the target
        clouds tx, tv (R, m, 3): an (R, count) array."""
        R, m = tx.shape[0], tx.shape[1]
        TY = torch.as_tensor(np.ascontiguousarray(tx.transpose(2, 0, 1).reshape(3, R * m)),
                             device=self.dev)
        TV = torch.as_tensor(np.ascontiguousarray(tv.transpose(2, 0, 1).reshape(3, R * m)),
                             device=self.dev)
        out = torch.empty(R * count, dtype=torch.float64, device=self.dev)
        nb.nbody_mmd_eval_cross(self.mmd, count, self.CX, self.CV, R, m, TY, TV, out)
        return out.cpu().numpy().reshape(R, count)

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


KMS = 1.0227121650537077e-3   # 1 km/s in kpc/Myr


def run(n=1000, steps=1000, t_end=500.0, per_dim=10, batch=1024, refine_iters=10,
        sigmas=(0.5, 1.0, 2.0), f_obs=(1.1, 0.9, 1.15, 0.85), width=0.3, seed=1,
        device="cuda:0", tuning=None, bootstrap=0, bootstrap_refine=0, sigma_frac=0.05,
        sigma_x=None, sigma_v_kms=None, refine_batch=512):
    cfg = dataclasses.replace(C1, n=n, n_steps=steps, t_acc=float(t_end))
    centre = np.array(cfg.theta_true, float)
    theta_obs = centre * np.array(f_obs)
    xh, vh = plummer_unit(n, seed)
    obs = StreamModel(cfg, xh, vh, device=device)
    tx, tv = obs.final_state(list(theta_obs))
    obs.close()
    grid = regular_grid(centre, width, per_dim)
    gs = GridSearch(cfg, xh, vh, tx, tv, sigmas=sigmas, batch=batch, device=device,
                    tuning=tuning, keep_clouds=len(grid) if bootstrap else 0)
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
    reals = None
    if bootstrap:
        # the observation redrawn from its errors, every kept cloud scored
        # against every realisation in one call
        ox = tx.cpu().numpy().T if hasattr(tx, "cpu") else np.asarray(tx).T
        ov = tv.cpu().numpy().T if hasattr(tv, "cpu") else np.asarray(tv).T
        # errors: given in kpc and km/s, else a fraction of the observed
        # cloud's spread in each coordinate
        ex = sigma_x if sigma_x is not None else sigma_frac * ox.std(axis=0)
        ev = sigma_v_kms * KMS if sigma_v_kms is not None else sigma_frac * ov.std(axis=0)
        rx, rv = perturbed_clouds(ox, ov, ex, ev, bootstrap, seed + 1000)
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        LB = gs.cross_losses(len(grid), rx, rv)
        t_b = time.perf_counter() - t0
        kb = np.argmin(LB, axis=1)
        bt = grid[kb]
        rel = bt / theta_obs[None, :] - 1.0
        pairs = float(len(grid)) * bootstrap * n * n
        res["bootstrap"] = {
            "realisations": bootstrap,
            "sigma_x_kpc": np.broadcast_to(ex, (3,)).tolist(),
            "sigma_v_kms": (np.broadcast_to(ev, (3,)) / KMS).tolist(),
            "time_s": t_b, "cloud_pairs_per_s": len(grid) * bootstrap / t_b,
            "kernel_pairs_per_s": pairs / t_b,
            "best_theta_mean": bt.mean(axis=0).tolist(),
            "best_theta_std": bt.std(axis=0).tolist(),
            "best_rel_err_mean": rel.mean(axis=0).tolist(),
            "distinct_best_points": int(len(np.unique(kb))),
            "fraction_at_noise_free_best": float(np.mean(kb == k))}
        reals = (rx, rv, bt)
    obs_scale = nb.nbody_mmd_target_stats(gs.mmd)[1]   # the observation's units
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
    if reals is not None and bootstrap_refine > 0:
        # gradient refinement of the first realisations, `refine_batch` at a
        # time: one batched pipeline (every member against its own
        # realisation) and one gradient call for all members per iteration
        rx, rv, bt = reals
        K = min(bootstrap_refine, bootstrap)
        est = np.empty((K, 4))
        t0 = time.perf_counter()
        for r0 in range(0, K, refine_batch):
            r1 = min(K, r0 + refine_batch)
            model = StreamBatch(cfg, xh, vh, rx[r0:r1], rv[r0:r1], sigmas, scale=obs_scale,
                                device=device)
            est[r0:r1], _, _ = descend_batch(model, bt[r0:r1], centre, width,
                                             iters=refine_iters)
            model.close()
        t_r = time.perf_counter() - t0
        res["bootstrap"]["refine"] = {
            "realisations": K, "iters": refine_iters, "batch": refine_batch, "time_s": t_r,
            "s_per_realisation": t_r / K, "theta_mean": est.mean(axis=0).tolist(),
            "theta_std": est.std(axis=0).tolist(),
            "rel_err_mean": (est / theta_obs[None, :] - 1.0).mean(axis=0).tolist()}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1000)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--t-end", type=float, default=500.0)
    ap.add_argument("--per-dim", type=int, default=10)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--refine", type=int, default=10)
    ap.add_argument("--bootstrap", type=int, default=0)
    ap.add_argument("--bootstrap-refine", type=int, default=0)
    ap.add_argument("--sigma-frac", type=float, default=0.05,
                    help="errors as a fraction of the observed spread per coordinate")
    ap.add_argument("--sigma-x", type=float, default=None, help="position error, kpc")
    ap.add_argument("--sigma-v", type=float, default=None, help="velocity error, km/s")
    ap.add_argument("--refine-batch", type=int, default=512,
                    help="realisations refined together (72 MB of trajectory each)")
    a = ap.parse_args()
    from . import build
    build.build()
    print(json.dumps(run(n=a.n, steps=a.steps, t_end=a.t_end, per_dim=a.per_dim,
                         batch=a.batch, refine_iters=a.refine, bootstrap=a.bootstrap,
                         bootstrap_refine=a.bootstrap_refine, sigma_frac=a.sigma_frac,
                         sigma_x=a.sigma_x,
                         sigma_v_kms=a.sigma_v, refine_batch=a.refine_batch)))


if __name__ == "__main__":
    main()

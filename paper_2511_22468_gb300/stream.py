"""Mock-stream inference on the GPU: the pipeline of the paper's Fig. 2 with
a binned-density loss or the paper's point-cloud (MMD) loss, and its
gradient as a torch.autograd.Function.

StreamModel owns one nbody_stream (C ABI); StreamLoss.apply(theta, model)
returns the loss as a tensor whose backward runs the discrete adjoint
(head, n-body reverse sweep, Plummer shift, backward orbit) in the
library's kernels.  theta = (t_end [Myr], M_Plummer, M_NFW, M_MN [Msun]).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import nbody as nb


# device memory the adjoint tape of one stream run may take before the run
# is split into recomputed segments (bytes)
TAPE_BUDGET = 16e9


def tape_interval(n, n_steps, budget=TAPE_BUDGET):
    """Checkpoint interval K for the stream run: the whole run as one kept
    segment (K = n_steps: the reverse sweep recomputes nothing) when its
    tape -- positions, accelerations and half-step velocities of every
    step, 72 bytes per (padded) particle and step -- fits the budget, else
    about sqrt(n_steps) steps per recomputed segment."""
    npad = -(-int(n) // 1024) * 1024
    if 72.0 * npad * n_steps <= budget:
        return int(n_steps)
    return max(1, int(round(math.sqrt(n_steps))))


def stream_cfg(cfg, n=None, n_steps=None, checkpoint_every=None) -> nb.nbody_stream_cfg:
    """C config from a StreamC1-like dataclass (configs.py)."""
    c = nb.nbody_stream_cfg()
    c.n = int(cfg.n if n is None else n)
    c.n_steps = int(cfg.n_steps if n_steps is None else n_steps)
    K = checkpoint_every or tape_interval(c.n, c.n_steps)
    c.checkpoint_every = int(K)
    c.G, c.eps, c.a_prog = cfg.G, cfg.eps, cfg.a_prog
    c.nfw_rs, c.mn_a, c.mn_b = cfg.pot.nfw_rs, cfg.pot.mn_a, cfg.pot.mn_b
    c.X0[:] = list(cfg.X0)
    c.V0[:] = list(cfg.V0)
    c.observer[:] = list(cfg.observer)
    c.nb1, c.nb2 = cfg.nb1, cfg.nb2
    c.phi1_lo, c.phi1_hi = (math.radians(a) for a in cfg.phi1_deg)
    c.phi2_lo, c.phi2_hi = (math.radians(a) for a in cfg.phi2_deg)
    return c


class StreamModel:
    def __init__(self, cfg, xhat, vhat, n_steps=None, checkpoint_every=None,
                 device="cuda:0", stream=None):
        xhat = np.asarray(xhat, np.float64)
        vhat = np.asarray(vhat, np.float64)
        self.n = xhat.shape[0]
        self.cfg = stream_cfg(cfg, n=self.n, n_steps=n_steps,
                              checkpoint_every=checkpoint_every)
        self.device = torch.device(device)
        xh = torch.tensor(xhat.T.copy(), device=self.device)
        vh = torch.tensor(vhat.T.copy(), device=self.device)
        if stream is not None:   # the copies above run on the caller's stream
            torch.cuda.current_stream(self.device).synchronize()
        self.h = nb.nbody_stream_create(self.cfg, xh, vh, stream)
        self.nb = (self.cfg.nb1, self.cfg.nb2)

    def close(self):
        if self.h is not None and self.h.value:
            nb.nbody_stream_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def density(self, theta):
        rho = torch.empty(self.nb, dtype=torch.float64, device=self.device)
        nb.nbody_stream_forward(self.h, theta, rho)
        return rho

    def set_target(self, target):
        t = torch.as_tensor(target, dtype=torch.float64).to(self.device).contiguous()
        nb.nbody_stream_set_target(self.h, t)

    def set_target_cloud(self, x, v, sigmas=(0.5, 1.0, 2.0), scale=None):
        """MMD^2 loss against the phase-space cloud x, v ((3, m) FP64
        tensors or arrays)."""
        tx = torch.as_tensor(x, dtype=torch.float64).to(self.device).contiguous()
        tv = torch.as_tensor(v, dtype=torch.float64).to(self.device).contiguous()
        nb.nbody_stream_set_target_cloud(self.h, tx, tv, list(sigmas), scale)

    def final_state(self, theta):
        """(x_T, v_T), (3, n) each, of the simulated stream at theta."""
        x0 = torch.empty((3, self.n), dtype=torch.float64, device=self.device)
        v0 = torch.empty_like(x0)
        m = torch.empty(self.n, dtype=torch.float64, device=self.device)
        com = nb.nbody_stream_initial_state(self.h, theta, x0, v0, m)
        p = self.cfg
        params = nb.make_params(p.G, p.eps, theta[0] / p.n_steps, ext_flags=3, nfw_M=theta[2],
                                nfw_rs=p.nfw_rs, mn_M=theta[3], mn_a=p.mn_a, mn_b=p.mn_b,
                                center=com[:3], center_vel=com[3:6],
                                center_mode=nb.NBODY_CENTER_GUIDE)
        sim = nb.Simulation(self.n, params)
        sim.set_state(x0, v0, m)
        xT, vT = torch.empty_like(x0), torch.empty_like(v0)
        sim.integrate(p.n_steps, xT, vT)
        sim.close()
        return xT, vT

    def loss(self, theta):
        return nb.nbody_stream_forward(self.h, theta)

    def grad(self):
        return nb.nbody_stream_grad(self.h)

    def autotune(self, theta, probe_launches=3):
        """Tune the n-body kernels' launch shapes on the state at theta."""
        nb.nbody_stream_autotune(self.h, theta, probe_launches)

    def loss_and_grad(self, theta):
        L = self.loss(theta)
        return L, np.array(self.grad())


class StreamBatch:
    """The point-cloud pipeline for many parameter vectors at once: member
    b's final cloud against its own target cloud b (targets: (count, m, 3)
    positions and velocities), all in the units `scale` (6 standard
    deviations) with the bandwidths `sigmas`."""

    def __init__(self, cfg, xhat, vhat, targets_x, targets_v, sigmas=(0.5, 1.0, 2.0),
                 scale=None, n_steps=None, device="cuda:0"):
        xhat = np.asarray(xhat, np.float64)
        vhat = np.asarray(vhat, np.float64)
        tx = np.asarray(targets_x, np.float64)
        tv = np.asarray(targets_v, np.float64)
        self.n = xhat.shape[0]
        self.count, m = tx.shape[0], tx.shape[1]
        self.cfg = stream_cfg(cfg, n=self.n, n_steps=n_steps)
        self.device = torch.device(device)
        if scale is None:   # the first target's spread
            scale = np.concatenate([tx[0].std(axis=0), tv[0].std(axis=0)])
        TX = torch.tensor(tx.transpose(2, 0, 1).reshape(3, self.count * m).copy(),
                          device=self.device)
        TV = torch.tensor(tv.transpose(2, 0, 1).reshape(3, self.count * m).copy(),
                          device=self.device)
        xh = torch.tensor(xhat.T.copy(), device=self.device)
        vh = torch.tensor(vhat.T.copy(), device=self.device)
        torch.cuda.current_stream(self.device).synchronize()
        self.h = nb.nbody_stream_batch_create(self.cfg, self.count, xh, vh, m, TX, TV,
                                              list(scale), list(sigmas))

    def loss_and_grad(self, thetas):
        """(losses (count,), dL/dtheta (count, 4)) at thetas (count, 4)."""
        return nb.nbody_stream_batch_loss_grad(self.h, thetas)

    def loss(self, thetas):
        return nb.nbody_stream_batch_loss_grad(self.h, thetas, want_grad=False)[0]

    def grad_parts(self):
        """(count, 2, 4): the two parts of every gradient component of the
        last loss_and_grad (n-body run / velocity scaling, orbit / masses)."""
        return nb.nbody_stream_batch_grad_parts(self.h, self.count)

    def close(self):
        if self.h is not None and self.h.value:
            nb.nbody_stream_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StreamLoss(torch.autograd.Function):
    """L(theta) with d L / d theta from the library's adjoint kernels."""

    @staticmethod
    def forward(ctx, theta, model: StreamModel):
        L = model.loss([float(t) for t in theta.detach().cpu().tolist()])
        ctx.model = model
        return torch.tensor(L, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, g):
        tb = torch.tensor(ctx.model.grad(), dtype=torch.float64, device=g.device)
        return tb * g, None


def horizon_sweep(horizons_myr=(50, 100, 200, 400, 800, 1600, 3000), rel=0.02,
                  seed=None, n=None):
    """Gradient of the stream loss against the accretion time horizon.

    For each horizon t (steps of 0.5 Myr), the target is the density at the
    true parameters and the gradient is taken at theta_true * (1 + rel).
    Returns rows (t, steps, loss, grad, smooth_scale) where smooth_scale =
    2 L / (rel t) is the size dL/dt_end would have if the loss were a smooth
    quadratic bowl around the truth; a gradient far above it is dominated by
    the exponential growth of the chaotic cluster's adjoint."""
    import dataclasses

    from .configs import C1
    from .inputs import plummer_unit
    xh, vh = plummer_unit(C1.n if n is None else n, C1.seed if seed is None else seed)
    rows = []
    for t in horizons_myr:
        ns = int(round(t / 0.5))
        cfg = dataclasses.replace(C1, t_acc=float(t), n_steps=ns)
        m = StreamModel(cfg, xh, vh)
        truth = np.array(cfg.theta_true, float)
        m.set_target(m.density(truth))
        L, g = m.loss_and_grad(truth * (1.0 + rel))
        rows.append((t, ns, L, list(g), 2.0 * L / (rel * t)))
        m.close()
    return rows


def time_pipeline(reps=3, autotune=True):
    """Seconds per loss (forward) and per gradient (reverse sweep, Plummer
    shift and orbit adjoints) of the stream workload (N = 1e4, 6000 steps of
    0.5 Myr), at theta_true * 1.02 with the target at theta_true."""
    import time

    from .configs import C1
    from .inputs import plummer_unit
    xh, vh = plummer_unit(C1.n, C1.seed)
    m = StreamModel(C1, xh, vh)
    truth = np.array(C1.theta_true, float)
    m.set_target(m.density(truth))
    th = list(truth * 1.02)
    if autotune:
        nb.nbody_stream_autotune(m.h, th)
    m.loss(th)
    m.grad()
    fw, gr = [], []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        L = m.loss(th)
        t1 = time.perf_counter()
        m.grad()
        t2 = time.perf_counter()
        fw.append(t1 - t0)
        gr.append(t2 - t1)
    shapes = {"pair": list(nb.nbody_stream_get_pair_shape(m.h, 0)),
              "vjp": list(nb.nbody_stream_get_pair_shape(m.h, 1))}
    m.close()
    return {"workload": "stream_n1e4_6000_steps", "forward_s": min(fw), "gradient_s": min(gr),
            "forward_us_per_step": 1e6 * min(fw) / C1.n_steps,
            "gradient_us_per_step": 1e6 * min(gr) / C1.n_steps, "loss": L, "shapes": shapes}


if __name__ == "__main__":
    import json
    import sys
    if "--time" in sys.argv:
        print(json.dumps(time_pipeline()), flush=True)
    if "--horizon-sweep" in sys.argv:
        for row in horizon_sweep():
            print(json.dumps({"t_end_myr": row[0], "steps": row[1], "loss": row[2],
                              "grad": row[3], "smooth_dLdt_scale": row[4]}), flush=True)

"""Learned warm start for stream inference (paper Sec. 3 outlook: a neural
network coupled to the differentiable solver).

  EnsembleDensities  -- binned stream densities for many parameter vectors:
                        initial states from the pipeline's orbit kernels, the
                        n-body runs as one batch (one persistent pair launch
                        per step for every member, graph-captured), the
                        density head per member; all in the library's kernels.
  Surrogate          -- the 4 -> 256 -> 256 -> 1024 GELU network trained and
                        evaluated by the library's kernels (nbody_mlp_*).
  descend            -- gradient descent on the simulator's loss with the
                        discrete-adjoint gradient (nbody_stream_grad): the
                        simulator supplies every final parameter.

Parameters are handled in normalised coordinates u = (theta / theta_c - 1)
/ width around a prior centre theta_c; the network maps u to 1024 * density
(unit mean per bin).
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import nbody as nb
from .stream import StreamModel

DENSITY_SCALE = 1024.0


def to_u(theta, centre, width):
    return (np.asarray(theta, float) / np.asarray(centre, float) - 1.0) / width


def from_u(u, centre, width):
    return np.asarray(centre, float) * (1.0 + width * np.asarray(u, float))


class EnsembleDensities:
    """Densities of one stream workload for many parameter vectors."""

    def __init__(self, cfg, xhat, vhat, batch=128, device="cuda:0", tuning=None):
        """batch simulations per persistent launch; tuning: a batch launch
        candidate, or None to time the candidates on the first batch's state
        (128 members with the tuned candidate and the batch's initial states
        from one batched call: 3.9 s per 512 simulations of N = 1e4 over 200
        steps on GB300, against 4.8 s for 64 untuned members set up one by
        one)."""
        self.dev = torch.device(device)
        self.cfg = cfg
        self.model = StreamModel(cfg, xhat, vhat, device=device)
        self.n = self.model.n
        self.B = batch
        self.steps = cfg.n_steps
        n, B = self.n, batch
        offs = np.arange(B + 1) * n
        self.h = nb.nbody_create_batch(offs, [self._params(cfg.theta_true, (0,) * 6)] * B)
        if tuning is not None:
            nb.nbody_set_tuning(self.h, tuning)
        self.tune_pending = tuning is None
        self.X = torch.empty((3, B * n), dtype=torch.float64, device=self.dev)
        self.V = torch.empty_like(self.X)
        self.M = torch.empty(B * n, dtype=torch.float64, device=self.dev)
        self.XO = torch.empty_like(self.X)
        self.xs = torch.empty((3, n), dtype=torch.float64, device=self.dev)

    def _params(self, th, com):
        c, p = self.cfg, self.cfg.pot
        return nb.make_params(c.G, c.eps, th[0] / c.n_steps, ext_flags=3, nfw_M=th[2],
                              nfw_rs=p.nfw_rs, mn_M=th[3], mn_a=p.mn_a, mn_b=p.mn_b,
                              center=com[:3], center_vel=com[3:6],
                              center_mode=nb.NBODY_CENTER_GUIDE)

    def densities(self, thetas):
        thetas = np.asarray(thetas, float)
        out = np.empty((len(thetas), self.cfg.nb1 * self.cfg.nb2))
        n, B = self.n, self.B
        rho = torch.empty(self.cfg.nb1 * self.cfg.nb2, dtype=torch.float64, device=self.dev)
        com = np.empty((B, 6))
        for c0 in range(0, len(thetas), B):
            chunk = thetas[c0:c0 + B]
            # the last vector repeats to fill a short final batch
            full = np.ascontiguousarray([chunk[min(j, len(chunk) - 1)] for j in range(B)])
            # backward orbits and Plummer shifts of the whole batch, written
            # straight into the batch layout (member j in columns j n ..)
            nb.nbody_stream_initial_states(self.model.h, full, self.X, self.V, self.M, com)
            prm = [self._params(full[j], com[j]) for j in range(B)]
            nb.nbody_set_params_batch(self.h, prm)
            nb.nbody_set_state(self.h, self.X, self.V, self.M)
            if self.tune_pending:  # times the candidates; the state is not advanced
                nb.nbody_autotune(self.h, 2)
                self.tune_pending = False
            nb.nbody_integrate(self.h, self.steps)
            nb.nbody_get_state(self.h, self.XO, None)
            for j in range(len(chunk)):
                self.xs.copy_(self.XO[:, j * n:(j + 1) * n])
                nb.nbody_stream_head(self.model.h, self.xs, rho)
                out[c0 + j] = rho.cpu().numpy()
        return out

    def close(self):
        if self.h is not None:
            nb.nbody_destroy(self.h)
            self.h = None
        self.model.close()


class Surrogate:
    def __init__(self, n_in=4, hidden=256, n_out=1024, max_batch=256, seed=0,
                 device="cuda:0"):
        self.dev = torch.device(device)
        self.dims = (n_in, hidden, n_out)
        self.max_batch = max_batch
        self.h = nb.nbody_mlp_create(n_in, hidden, n_out, max_batch)
        rng = np.random.default_rng(seed)
        # He-style initial weights, zero biases (random numbers drawn here,
        # passed to the library)
        P = [rng.normal(size=(hidden, n_in)) * np.sqrt(2.0 / n_in), np.zeros(hidden),
             rng.normal(size=(hidden, hidden)) * np.sqrt(2.0 / hidden), np.zeros(hidden),
             rng.normal(size=(n_out, hidden)) * np.sqrt(1.0 / hidden), np.zeros(n_out)]
        flat = np.concatenate([p.reshape(-1) for p in P]).astype(np.float32)
        nb.nbody_mlp_set_params(self.h, flat)

    def fit(self, U, Y, epochs=200, lr=1e-3, batch=256, U_val=None, Y_val=None, seed=0,
            log_every=20):
        U = torch.tensor(np.asarray(U, np.float32), device=self.dev)
        Y = torch.tensor(np.asarray(Y, np.float32), device=self.dev)
        n = U.shape[0]
        rng = np.random.default_rng(seed)
        hist = []
        for ep in range(epochs):
            perm = torch.tensor(rng.permutation(n), device=self.dev)
            last = None
            for b0 in range(0, n - batch + 1, batch):
                idx = perm[b0:b0 + batch]
                ub = U.index_select(0, idx).contiguous()
                yb = Y.index_select(0, idx).contiguous()
                want = (b0 + 2 * batch > n) and (ep % log_every == 0 or ep == epochs - 1)
                last = nb.nbody_mlp_loss_grad(self.h, ub, yb, want_loss=want)
                nb.nbody_mlp_adam_step(self.h, lr)
            if ep % log_every == 0 or ep == epochs - 1:
                row = {"epoch": ep, "train_mse": last}
                if U_val is not None:
                    row["val_mse"] = self.mse(U_val, Y_val)
                hist.append(row)
        self.check()
        return hist

    def check(self):
        """Raise if a tensor-core GEMM of the network gave up waiting."""
        rc = nb.nbody_mlp_get_status(self.h)
        if rc != nb.NBODY_OK:
            raise nb.NBodyError(rc, "surrogate network")

    def predict(self, U):
        U = torch.tensor(np.asarray(U, np.float32), device=self.dev)
        out = []
        for b0 in range(0, U.shape[0], self.max_batch):
            ub = U[b0:b0 + self.max_batch].contiguous()
            y = torch.empty((ub.shape[0], self.dims[2]), dtype=torch.float32, device=self.dev)
            nb.nbody_mlp_forward(self.h, ub, y)
            out.append(y.cpu().numpy())
        return np.concatenate(out)

    def mse(self, U, Y):
        return float(np.mean((self.predict(U) - np.asarray(Y)) ** 2))

    def invert(self, y_obs, starts=64, iters=400, lr=0.05, seed=0, lo=-1.5, hi=1.5):
        """Best input for an observed (scaled) density, multi-start Adam."""
        rng = np.random.default_rng(seed)
        u = torch.tensor(rng.uniform(-1, 1, (starts, self.dims[0])).astype(np.float32),
                         device=self.dev)
        t = torch.tensor(np.asarray(y_obs, np.float32), device=self.dev)
        loss = torch.empty(starts, dtype=torch.float32, device=self.dev)
        nb.nbody_mlp_invert(self.h, t, u, iters, lr, lo, hi, loss)
        self.check()
        k = int(torch.argmin(loss).item())
        return u[k].cpu().numpy().astype(float), float(loss[k].item())

    def close(self):
        if self.h is not None:
            nb.nbody_mlp_destroy(self.h)
            self.h = None


def descend_batch(model, thetas0, centre, width, lr=0.05, iters=10):
    """descend() for many problems at once (a StreamBatch: one gradient call
    for all members per iteration): per member Adam in normalised
    parameters, a step that raises the member's loss above its best is
    undone, its moments reset and its rate halved; returns the minimum-loss
    iterate of every member (count, 4), its loss (count,) and the best loss
    after every iteration (iters + 1, count)."""
    centre = np.asarray(centre, float)
    u = to_u(thetas0, centre, width)
    count = u.shape[0]
    m = np.zeros_like(u)
    v = np.zeros_like(u)
    k = np.zeros(count)
    lr = np.full(count, float(lr))
    best_L = np.full(count, np.inf)
    best_u = u.copy()
    best_g = np.zeros_like(u)
    trace = []
    for it in range(iters + 1):
        L, g = model.loss_and_grad(from_u(u, centre, width))
        gu = g * centre[None, :] * width
        better = L <= best_L
        best_L = np.where(better, L, best_L)
        best_u[better] = u[better]
        best_g[better] = gu[better]
        worse = ~better
        lr[worse] *= 0.5
        m[worse] = 0.0
        v[worse] = 0.0
        k[worse] = 0
        u[worse] = best_u[worse]
        gu[worse] = best_g[worse]
        trace.append(best_L.copy())
        if it == iters:
            break
        ok = np.all(np.isfinite(gu), axis=1)
        k += ok
        m[ok] = 0.9 * m[ok] + 0.1 * gu[ok]
        v[ok] = 0.999 * v[ok] + 0.001 * gu[ok] * gu[ok]
        kk = np.maximum(k, 1)[:, None]
        step = lr[:, None] * (m / (1 - 0.9 ** kk)) / (np.sqrt(v / (1 - 0.999 ** kk)) + 1e-300)
        u[ok] = np.clip(u[ok] - step[ok], -1.5, 1.5)
    return from_u(best_u, centre, width), best_L, np.array(trace)


def descend(model: StreamModel, theta0, centre, width, lr=0.05, max_iters=50,
            loss_target=None, theta_true=None, err_target=None, clock=None, grow=1.0,
            lr_max=None):
    """Gradient descent on the simulator's loss in normalised parameters u,
    with the discrete-adjoint gradient dL/du = dL/dtheta * theta_c * width.
    Adam steps from the current point; the estimate is the minimum-loss
    iterate (as in the paper's Fig. 2, step 5); a step that raises the loss
    above the best is undone, the moments reset and the rate halved.
    A step that lowers the loss multiplies the rate by `grow` (up to
    lr_max), so that a rate halved by a noisy step recovers.
    Stops at loss_target, at parameter error err_target
    (max_k |theta_k / theta_true_k - 1|) or after max_iters simulator
    gradients; each trajectory row holds the best iterate so far."""
    lr_max = lr if lr_max is None else lr_max
    clock = clock or time.perf_counter
    t0 = clock()
    u = to_u(theta0, centre, width)
    m = np.zeros(4)
    v = np.zeros(4)
    k = 0
    best = None
    traj = []
    for it in range(max_iters + 1):
        th = from_u(u, centre, width)
        L, g = model.loss_and_grad(th)
        gu = np.asarray(g) * np.asarray(centre) * width
        if best is None or L <= best[0]:
            if best is not None:
                lr = min(lr * grow, lr_max)
            best = (L, u.copy(), gu)
        else:
            lr *= 0.5
            m[:] = 0.0
            v[:] = 0.0
            k = 0
            u = best[1].copy()
            gu = best[2]
        Lb, ub = best[0], best[1]
        thb = from_u(ub, centre, width)
        err = None if theta_true is None else float(np.max(np.abs(thb / theta_true - 1.0)))
        traj.append({"iter": it, "t": clock() - t0, "loss": Lb, "loss_evaluated": L,
                     "theta": thb.tolist(), "err": err, "lr": lr})
        if (loss_target is not None and Lb <= loss_target) or \
                (err_target is not None and err is not None and err <= err_target):
            break
        if it == max_iters or not np.all(np.isfinite(gu)):
            break
        k += 1
        m = 0.9 * m + 0.1 * gu
        v = 0.999 * v + 0.001 * gu * gu
        u = np.clip(u - lr * (m / (1 - 0.9 ** k)) / (np.sqrt(v / (1 - 0.999 ** k)) + 1e-300),
                    -1.5, 1.5)
    return traj

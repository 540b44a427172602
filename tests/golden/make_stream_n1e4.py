"""Expected values of the mock-stream pipeline at the stream workload's own
particle number, computed by the FP64 oracle alone.

The GD-1-like stream workload (Fig. 2; Sec. 2.2.1) runs a Plummer
progenitor of N = 10^4 particles; at that size the oracle's reverse sweep
takes minutes, too long for a test, so this script writes its results once:

  * the target density at the true parameters Theta_true = (t_end, 2e4 Msun,
    1e12 Msun, 6.8e10 Msun), t_end = n_steps * 0.5 Myr;
  * at Theta = 1.1 Theta_true: the 32 x 32 density, the loss, dL/dTheta by
    the oracle's adjoint with the two parts of every component (the n-body
    run's and the backward orbit's), and dL/dTheta by Richardson-extrapolated
    central differences of the oracle's loss (relative steps 1e-4, 5e-5);
  * a fingerprint of the seeded unit Plummer sample the results belong to.

Only `oracle/` computes; `paper_2511_22468_gb300.inputs` draws the seeded
initial conditions and `configs` holds the workload's constants.

    python tests/golden/make_stream_n1e4.py [--steps 200]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import stream as ostream  # noqa: E402
from paper_2511_22468_gb300.configs import C1  # noqa: E402
from paper_2511_22468_gb300.inputs import plummer_unit  # noqa: E402

DT_MYR = 0.5
FACTORS = (1.1, 1.1, 1.1, 1.1)


def fingerprint(xh, vh):
    """Sums and sampled entries of the unit sample (compared to 1e-12)."""
    idx = [0, 1, len(xh) // 2, len(xh) - 1]
    return {"sum_abs_x": float(np.abs(xh).sum()), "sum_abs_v": float(np.abs(vh).sum()),
            "rows": idx, "x_rows": xh[idx].tolist(), "v_rows": vh[idx].tolist()}


def golden_path(steps):
    return os.path.join(HERE, "stream_n1e4_s%d.json" % steps)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=200)
    a = ap.parse_args()
    cfg = dataclasses.replace(C1, t_acc=a.steps * DT_MYR, n_steps=a.steps)
    xh, vh = plummer_unit(cfg.n, cfg.seed)
    orc = ostream.StreamModel(cfg, xh, vh)
    truth = np.array(cfg.theta_true, float)
    theta = truth * np.array(FACTORS)
    t0 = time.time()
    target = orc.density(truth)
    rho = orc.density(theta)
    L, g = orc.loss_and_grad(theta, target)
    parts = [list(map(float, p)) for p in orc.grad_parts]
    t_end_parts = [float(p) for p in orc.t_end_parts]
    fd = []
    for k in range(4):
        h = 1e-4 * theta[k]

        def f(s):
            t = theta.copy()
            t[k] += s
            return orc.loss(t, target)
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        fd.append((4 * d2 - d1) / 3)
    out = {
        "_about": "mock-stream pipeline (Fig. 2, Sec. 2.2.1) at N = 10^4, written by "
                  "tests/golden/make_stream_n1e4.py from the FP64 oracle",
        "n": cfg.n, "n_steps": cfg.n_steps, "t_end_true": cfg.t_acc, "seed": cfg.seed,
        "theta_true": truth.tolist(), "theta": theta.tolist(),
        "target_density": target.ravel().tolist(), "density": rho.ravel().tolist(),
        "loss": float(L), "grad": [float(t) for t in g], "grad_parts": parts,
        "t_end_parts": t_end_parts, "grad_fd_richardson": [float(t) for t in fd],
        "inputs": fingerprint(xh, vh), "oracle_seconds": time.time() - t0,
    }
    with open(golden_path(cfg.n_steps), "w") as fh:
        json.dump(out, fh, indent=0)
        fh.write("\n")
    print(golden_path(cfg.n_steps), "loss", L, "grad", g, "fd", fd,
          "%.0f s" % out["oracle_seconds"])


if __name__ == "__main__":
    main()

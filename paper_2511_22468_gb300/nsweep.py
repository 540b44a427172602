"""Throughput of one simulation against its particle number on one GPU (the
workload of the paper's Fig. 1: the tidal disruption of a Plummer sphere in
the Milky Way potential, there distributed over 1-5 GPUs).

For every N: a Plummer sphere of 2e4 M_sun (a = 10 pc, eps = 1 pc) at the
stream progenitor's phase-space point in NFW + Miyamoto-Nagai + bulge,
dt = 0.5 Myr; the pair-kernel launch shape is autotuned on the state, a
warm-up run captures the step loop as a CUDA graph, then `steps` steps are
timed with CUDA events (forward integration; the reverse sweep with
--adjoint).  Reported: ms per step, pair interactions per second (N^2 per
step), pair evaluations per second (a run of k kick-drift-kick steps makes
k + 1 pair passes: the kicks at both ends of a step share one force) and
the fraction of the FP32 peak at 20 flops per evaluation.

    python -m paper_2511_22468_gb300.nsweep [--sizes 1000,10000,...] [--adjoint] [--steps K]
        [--pair-shape V,T,R,S] [--vjp-shape V,T,R,S]
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import nbody as nb
from .configs import C1, G_KPC_MSUN_MYR
from .inputs import plummer_sphere

BULGE = dict(bulge_M=5e9, bulge_alpha=1.8, bulge_rc=1.9)


def peak_tflops(dev):
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    return sms * 128 * 2 * 2.07e9 / 1e12


def measure(n, steps, adjoint=False, device="cuda:0", seed=5, shapes=None):
    """One size; shapes = (pair, vjp) launch shapes (variant, threads,
    per_thread, chunks), either None, replaces the autotuner when given."""
    dev = torch.device(device)
    pot = C1.pot
    x, v, m = plummer_sphere(n, seed, G_KPC_MSUN_MYR, C1.M_prog, C1.a_prog, center=C1.X0,
                             velocity=C1.V0)
    p = nb.make_params(G_KPC_MSUN_MYR, C1.eps, 0.5, checkpoint_every=10 if adjoint else 0,
                       ext_flags=7, nfw_M=pot.nfw_M, nfw_rs=pot.nfw_rs, mn_M=pot.mn_M,
                       mn_a=pot.mn_a, mn_b=pot.mn_b, center=C1.X0, center_vel=C1.V0,
                       center_mode=nb.NBODY_CENTER_GUIDE, **BULGE)
    X = torch.tensor(x.T.copy(), device=dev)
    V = torch.tensor(v.T.copy(), device=dev)
    M = torch.tensor(m, device=dev)
    sim = nb.Simulation(n, p)
    sim.set_state(X, V, M)
    if shapes is None:
        fwd_shape, vjp_shape = nb.nbody_autotune_pair(sim.h)
    else:
        for vjp, sh in enumerate(shapes):
            if sh is not None:
                nb.nbody_set_pair_shape(sim.h, vjp, *sh)
        fwd_shape, vjp_shape = nb.nbody_get_pair_shape(sim.h, 0), nb.nbody_get_pair_shape(sim.h, 1)
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    sim.integrate(steps)                      # warm-up (captures the graph)
    if adjoint:
        sim.vjp(X, None)
    sim.set_state(X, V, M)
    torch.cuda.synchronize(dev)
    # the timed region is an NVTX range ("timed"), so that a profiler can be
    # limited to it and skip the autotuner's and the warm-up's launches
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    sim.integrate(steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_fwd = e0.elapsed_time(e1) / 1e3
    row = {"n": n, "steps": steps, "ms_per_step": 1e3 * t_fwd / steps,
           "interactions_per_s": float(n) * n * steps / t_fwd,
           "pair_evaluations_per_s": float(n) * n * (steps + 1) / t_fwd}
    row["pct_fp32_peak"] = 100.0 * 20.0 * row["pair_evaluations_per_s"] / 1e12 / peak_tflops(dev)
    if adjoint:
        torch.cuda.synchronize(dev)
        e0.record(stream)
        sim.vjp(X, None)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t_bwd = e0.elapsed_time(e1) / 1e3
        row["adjoint_ms_per_step"] = 1e3 * t_bwd / steps
        row["fwd_adjoint_interactions_per_s"] = 2.0 * n * n * steps / (t_fwd + t_bwd)
    torch.cuda.nvtx.range_pop()
    row["shapes"] = {"pair": list(fwd_shape), "vjp": list(vjp_shape)}
    row["status_ok"] = sim.status() == 0
    sim.close()
    return row


def default_steps(n):
    # about 2e11 pair interactions per size, at least 10 steps, at most 2000
    return int(min(2000, max(10, 2e11 / (float(n) * n))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", default="1000,3000,10000,30000,100000,300000,1000000")
    ap.add_argument("--adjoint", action="store_true")
    ap.add_argument("--steps", type=int, default=None,
                    help="steps per size (default: about 2e11 interactions)")
    ap.add_argument("--pair-shape", default=None,
                    help="variant,threads,per_thread,chunks of the pair-force kernel "
                         "(with --vjp-shape: instead of the autotuner)")
    ap.add_argument("--vjp-shape", default=None, help="the same for the pair-VJP kernel")
    a = ap.parse_args()
    from . import build
    build.build()
    shapes = None
    if a.pair_shape or a.vjp_shape:
        shapes = tuple(tuple(int(v) for v in sh.split(",")) if sh else None
                       for sh in (a.pair_shape, a.vjp_shape))
    for n in [int(s) for s in a.sizes.split(",")]:
        steps = a.steps if a.steps else default_steps(n)
        print(json.dumps(measure(n, steps, adjoint=a.adjoint, shapes=shapes)), flush=True)


if __name__ == "__main__":
    main()

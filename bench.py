#!/usr/bin/env python3
"""Throughput benchmark of the differentiable direct-sum N-body path.

Workload: an N = 1e6 Plummer sphere (1e6 Msun, a = 50 pc, eps = 0.5 pc) at
the stream progenitor's present-day phase-space point in the NFW + MN
potential, dt = 0.5 Myr, adjoint checkpoints every 10 steps, FP32 pair
interactions with FP64 state.  That job is 100 kick-drift-kick steps forward
plus the reverse sweep.  One benchmark step is one checkpoint segment of it:
nbody_integrate(10 steps) continuing the trajectory, then nbody_vjp over
those 10 steps with the lean tape (the segment is recomputed from its
checkpoint, as every segment but the last is in the full job).

value = fwd+adjoint pair interactions/s = 2 * N^2 * 10 / step time, summed
over ranks (independent replicas, one per GPU); the kernel-level forward
rate and the fraction of the FP32 CUDA-core peak are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("pair interactions/s (fwd, fwd+adjoint) at N=1e6 and % FP32 peak; "
          "batched sims/s")
UNIT = "interactions/s"
SEG = 10                  # KDK steps per benchmark step (= checkpoint spacing)
FLOPS_PAIR = 20           # flops per interaction, forward convention
FLOPS_VJP = 41            # flops per interaction of the pair VJP kernel
# flops the kernels execute per interaction (FADD = FMUL = rsqrt = 1,
# FFMA = 2).  Equal masses: force 3 FADD + 6 FFMA + 2 FMUL + rsqrt = 18,
# VJP 6 FADD + 11 FFMA + 5 FMUL + rsqrt = 34; general masses: force 19,
# VJP 41 (the convention's count is the general VJP's).
EXEC_FLOPS = {("pair", True): 18, ("pair", False): 19, ("vjp", True): 34, ("vjp", False): 41}
FP32_LANES = 128          # FP32 FMA lanes per SM
L2_BYTES = 129 * 2 ** 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    # end-to-end steps: by default as many as the timed device steps
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-grid", action="store_true")
    ap.add_argument("--no-stream", action="store_true")
    ap.add_argument("--no-recovery", action="store_true")
    # the grid search's bootstrap (1000 resampled observations) is opt-in
    ap.add_argument("--bootstrap", action="store_true")
    # particle number of the throughput workload; other values than the
    # default serve profiling captures of a smaller case and name their size
    # in config.workload
    ap.add_argument("--n", type=int, default=None)
    return ap.parse_args()


def aggregate(local_ms, local_units, world):
    """Whole-job throughput of independent replicas: the units every rank
    processed over the slowest rank's time.  Returns (max ms, units/s)."""
    import torch
    t = torch.tensor([float(local_ms), float(local_units)], dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist
        if dist.get_backend() == "nccl":
            t = t.cuda()
        tmax = t[:1].clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        tsum = t[1:].clone()
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        ms, units = float(tmax.item()), float(tsum.item())
    else:
        ms, units = float(local_ms), float(local_units)
    return ms, units / (ms / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_arrays(n=None):
    import dataclasses

    from paper_2511_22468_gb300.configs import C3
    from paper_2511_22468_gb300.inputs import plummer_sphere
    if n is not None and n != C3.n:
        C3 = dataclasses.replace(C3, n=int(n), name="plummer_n%d_nfw_mn" % int(n))
    x, v, m = plummer_sphere(C3.n, C3.seed, C3.G, C3.M, C3.a, center=C3.X0,
                             velocity=C3.V0)
    rng = np.random.default_rng(C3.seed + 1)
    xbar = rng.normal(size=x.shape)
    return C3, x, v, m, xbar


def config_json(C3):
    return {"workload": C3.name, "n": C3.n, "M_msun": C3.M, "a_kpc": C3.a,
            "eps_kpc": C3.eps, "dt_myr": C3.dt, "potential": "NFW+MN",
            "job_steps": C3.n_steps, "checkpoint_every": C3.checkpoint_every,
            "bench_step": "integrate %d KDK steps + vjp over them (lean tape: "
                          "segment recomputed)" % SEG,
            "interactions_per_step": "2*N^2*%d (fwd + adjoint)" % SEG,
            "l2": "inputs larger than L2: state + tape touched per step "
                  "%.1f GB > 129 MB" % ((48 + 72 * SEG + 72) * C3.n / 1e9)}


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), float(f[3]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[3][k].lower() == "active"})
        load = [r for r in rows if r[2] > 200.0] or rows
        return {"sm_mhz": statistics.median(r[0] for r in load),
                "sm_max_mhz": max(r[1] for r in rows),
                "power_w_median": statistics.median(r[2] for r in load),
                "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------ cpu baseline --
def oracle_sample(x, m, G, eps, rows_acc, rows_vjp, seed=0):
    """Time the FP64 oracle on a row sample of the pair force and pair VJP at
    full N; returns (seconds for one benchmark step's pair work, details)."""
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    from oracle import core as orc
    n = x.shape[0]
    rng = np.random.default_rng(seed)
    ra = np.sort(rng.choice(n, rows_acc, replace=False))
    rv = np.sort(rng.choice(n, rows_vjp, replace=False))
    lam = rng.normal(size=x.shape)
    t0 = time.perf_counter()
    orc.pair_accel(x, m, G, eps, rows=ra)
    ta = time.perf_counter() - t0
    t0 = time.perf_counter()
    orc.pair_vjp(x, m, G, eps, lam, rows=rv)
    tv = time.perf_counter() - t0
    # one benchmark step: SEG forward + (SEG-1) recomputed pair passes and
    # SEG+1 VJP passes over all N rows
    step_s = (2 * SEG - 1) * ta * n / rows_acc + (SEG + 1) * tv * n / rows_vjp
    return step_s, ta + tv


def cpu_cores():
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


# -------------------------------------------------------------- reference --
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    C3, x, v, m, _ = workload_arrays(args.n)
    from oracle.build import build_oracle
    build_oracle()
    ra, rv = 1024, 128
    n = C3.n
    for _ in range(args.warmup):
        oracle_sample(x, m, C3.G, C3.eps, ra, rv)
    steps = []
    wall = 0.0
    for k in range(args.steps):
        s, w = oracle_sample(x, m, C3.G, C3.eps, ra, rv, seed=k + 1)
        steps.append(s)
        wall += w
    step_s = float(np.mean(steps))
    value = 2.0 * n * n * SEG / step_s
    sample = ("per step: oracle pair force on %d and pair VJP on %d sampled rows "
              "against all N = %d, scaled to the %d forward + %d recomputed + %d "
              "VJP passes of one step" % (ra, rv, n, SEG, SEG - 1, SEG + 1))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_json(C3),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(),
                             "kind": "oracle", "sample": sample,
                             "wall_s": wall},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------- ensemble --
def ensemble_members():
    """The 64-simulation ensemble: N log-uniform in [2048, 32768], the four
    stream parameters uniform within +-30 % of the stream workload's, each a
    Plummer progenitor (a = 10 pc, eps = 1 pc) at the present-day point,
    dt = t_end / 6000."""
    from paper_2511_22468_gb300.configs import C1, C2
    from paper_2511_22468_gb300.inputs import (log_uniform_sizes, plummer_sphere,
                                               uniform_factors)
    sizes = log_uniform_sizes(C2.n_sims, C2.n_lo, C2.n_hi, C2.seed_sizes)
    fac = uniform_factors(C2.n_sims, C2.width, 4, C2.seed_params)
    truth = np.array(C1.theta_true)
    out = []
    for s in range(C2.n_sims):
        th = truth * fac[s]
        x, v, m = plummer_sphere(int(sizes[s]), C2.seed_ics + s, C1.G, th[1], C1.a_prog,
                                 center=C1.X0, velocity=C1.V0)
        out.append((x, v, m, th))
    return out


def measure_ensemble(dev, gpu_name, plain_subset=8, plain_steps=200):
    import torch
    from paper_2511_22468_gb300 import autotune, nbody as nb
    from paper_2511_22468_gb300.configs import C1, C2
    mem = ensemble_members()
    pot = C1.pot

    def prm(th):
        return nb.make_params(C1.G, C1.eps, th[0] / C2.steps_per_t_acc, ext_flags=3,
                              nfw_M=th[2], nfw_rs=pot.nfw_rs, mn_M=th[3], mn_a=pot.mn_a,
                              mn_b=pot.mn_b, center=C1.X0, center_vel=C1.V0,
                              center_mode=nb.NBODY_CENTER_GUIDE)
    sizes = [x.shape[0] for x, _, _, _ in mem]
    offs = np.cumsum([0] + sizes)
    X = torch.tensor(np.concatenate([a[0] for a in mem]).T.copy(), device=dev)
    V = torch.tensor(np.concatenate([a[1] for a in mem]).T.copy(), device=dev)
    M = torch.tensor(np.concatenate([a[2] for a in mem]), device=dev)
    stream = torch.cuda.current_stream(dev)
    h = nb.nbody_create_batch(offs, [prm(a[3]) for a in mem], stream)
    nb.nbody_set_state(h, X, V, M)
    choice, src, ms = autotune.tune(h, sizes, gpu_name, probe_steps=2)
    steps = C2.n_steps
    nb.nbody_integrate(h, steps)            # captures the graph, warm-up
    nb.nbody_set_state(h, X, V, M)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    nb.nbody_integrate(h, steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t = e0.elapsed_time(e1) / 1e3
    ok = nb.nbody_get_status(h) == 0
    nb.nbody_destroy(h)
    inter = float(np.sum(np.asarray(sizes, float) ** 2)) * steps

    # the same members, a subset, one simulation per launch sequence (each
    # with the launch shapes tuned for its size, untimed) vs batched
    idx = np.argsort(sizes)[:: max(1, len(sizes) // plain_subset)][:plain_subset]
    sub = [mem[k] for k in idx]
    t_plain = 0.0
    for x, v, m, th in sub:
        sim = nb.Simulation(x.shape[0], prm(th), stream)
        sim.set_state(torch.tensor(x.T.copy(), device=dev), torch.tensor(v.T.copy(), device=dev),
                      torch.tensor(m, device=dev))
        nb.nbody_autotune_pair(sim.h)
        sim.step(5)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        sim.step(plain_steps)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t_plain += e0.elapsed_time(e1) / 1e3
        sim.close()
    so = np.cumsum([0] + [a[0].shape[0] for a in sub])
    hb = nb.nbody_create_batch(so, [prm(a[3]) for a in sub], stream)
    nb.nbody_set_state(hb, torch.tensor(np.concatenate([a[0] for a in sub]).T.copy(), device=dev),
                       torch.tensor(np.concatenate([a[1] for a in sub]).T.copy(), device=dev),
                       torch.tensor(np.concatenate([a[2] for a in sub]), device=dev))
    nb.nbody_set_tuning(hb, choice)
    nb.nbody_integrate(hb, plain_steps)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    nb.nbody_integrate(hb, plain_steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    t_batch_sub = e0.elapsed_time(e1) / 1e3
    nb.nbody_destroy(hb)
    return {"workload": C2.name, "n_sims": len(sizes), "steps": steps,
            "sizes_min_max": [int(min(sizes)), int(max(sizes))],
            "seconds_per_run": t, "sims_per_s": len(sizes) / t,
            "interactions_per_s": inter / t, "status_ok": ok,
            "tuning": {"choice": choice, "source": src, "ms_per_candidate": ms},
            "plain_vs_batched_subset": {
                "sims": plain_subset, "steps": plain_steps,
                "sizes": [int(mem[k][0].shape[0]) for k in idx],
                "plain_s": t_plain, "batched_s": t_batch_sub,
                "speedup": t_plain / t_batch_sub}}


# ------------------------------------------------------- stream workload --
def measure_stream_c1(dev, peak_max):
    """The GD-1-like stream workload at its own size (N = 10^4, 6000 steps
    of 0.5 Myr): seconds per loss and per gradient of the whole pipeline
    (launch shapes autotuned), as microseconds per step, and the pair
    kernels alone on the progenitor at N = 10^4 (tuned shape, CUDA-event
    timing of each launch)."""
    import torch
    from paper_2511_22468_gb300 import nbody as nb
    from paper_2511_22468_gb300.configs import C1
    from paper_2511_22468_gb300.inputs import plummer_sphere
    from paper_2511_22468_gb300.stream import time_pipeline
    t = time_pipeline(reps=2, autotune=True)
    out = {"workload": "gd1_stream_n10k_6000_steps", "forward_s": t["forward_s"],
           "gradient_s": t["gradient_s"], "forward_us_per_step": t["forward_us_per_step"],
           "fwd_adjoint_us_per_step": t["forward_us_per_step"] + t["gradient_us_per_step"],
           "pipeline_shapes": t.get("shapes")}
    n, steps = C1.n, 200
    x, v, m = plummer_sphere(n, C1.seed, C1.G, C1.M_prog, C1.a_prog, center=C1.X0,
                             velocity=C1.V0)
    pot = C1.pot
    prm = nb.make_params(C1.G, C1.eps, 0.5, checkpoint_every=10, ext_flags=3,
                         nfw_M=pot.nfw_M, nfw_rs=pot.nfw_rs, mn_M=pot.mn_M, mn_a=pot.mn_a,
                         mn_b=pot.mn_b, center=C1.X0, center_vel=C1.V0,
                         center_mode=nb.NBODY_CENTER_GUIDE, tape_mode=nb.NBODY_TAPE_LEAN)
    sim = nb.Simulation(n, prm)
    X = torch.tensor(x.T.copy(), device=dev)
    sim.set_state(X, torch.tensor(v.T.copy(), device=dev), torch.tensor(m, device=dev))
    fwd_shape, vjp_shape = nb.nbody_autotune_pair(sim.h)
    nb.nbody_set_timing(sim.h, True)
    sim.integrate(steps)
    sim.vjp(X, None)
    kt = nb.nbody_kernel_times(sim.h)
    for name, flops, shape in (("pair", FLOPS_PAIR, fwd_shape), ("vjp", FLOPS_VJP, vjp_shape)):
        ms, cnt = kt[name]
        avg = ms / cnt / 1e3
        ach = flops * n * n / avg / 1e12
        out[name + "_kernel"] = {"avg_us": avg * 1e6, "launches": cnt,
                                 "interactions_per_s": n * n / avg,
                                 "flops_per_interaction": flops,
                                 "frac_of_peak_at_2070MHz": ach / peak_max,
                                 "executed_flops_per_interaction": EXEC_FLOPS[(name, True)],
                                 "frac_executed_of_peak_at_2070MHz":
                                     ach * EXEC_FLOPS[(name, True)] / flops / peak_max,
                                 "shape": list(shape)}
    sim.close()
    return out


# ------------------------------------------------------------------- ours --
def hbm_peak():
    """Measured copy bandwidth of the GB300s (GB/s), else the
    profiling recipe's fallback."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def kernel_source_hash(src):
    """First 16 hex digits of the SHA-256 of a kernel's source file followed
    by the device-code headers it includes (in include order; the shared
    declarations header nbody_internal.cuh holds no device code and is left
    out), so that a change to the kernel's code voids the recorded counters."""
    csrc = os.path.join(ROOT, "paper_2511_22468_gb300", "csrc")
    text = open(os.path.join(csrc, src), "rb").read()
    h = hashlib.sha256(text)
    for line in text.decode().splitlines():
        line = line.strip()
        if line.startswith('#include "'):
            inc = os.path.join(csrc, line.split('"')[1])
            if os.path.exists(inc) and not inc.endswith("nbody_internal.cuh"):
                h.update(open(inc, "rb").read())
    return h.hexdigest()[:16]


def traffic_record(kernel):
    """Per-launch DRAM traffic of a kernel from the committed ncu summary,
    valid only while the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    src = {"pair": "pair_force.cu", "vjp": "pair_vjp.cu"}.get(kernel)
    if src is None:
        return None
    h = kernel_source_hash(src)
    for line in open(path):
        kv = dict(t.split("=", 1) for t in line.split() if "=" in t)
        if kv.get("kernel") == kernel and kv.get("source_sha256_16") == h:
            return float(kv["bytes_per_launch"])
    return None


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2511_22468_gb300 import build, nbody as nb
    build.build()
    C3, x, v, m, xbar = workload_arrays(args.n)
    n = C3.n
    p = C3.pot
    prm = nb.make_params(C3.G, C3.eps, C3.dt, checkpoint_every=SEG, ext_flags=3,
                         nfw_M=p.nfw_M, nfw_rs=p.nfw_rs, mn_M=p.mn_M, mn_a=p.mn_a,
                         mn_b=p.mn_b, center=C3.X0, center_vel=C3.V0,
                         center_mode=nb.NBODY_CENTER_GUIDE,
                         tape_mode=nb.NBODY_TAPE_LEAN)
    X = torch.tensor(x.T.copy(), device=dev)
    V = torch.tensor(v.T.copy(), device=dev)
    M = torch.tensor(m, device=dev)
    XB = torch.tensor(xbar.T.copy(), device=dev)
    X0B = torch.empty_like(X)
    V0B = torch.empty_like(X)
    stream = torch.cuda.current_stream(dev)
    sim = nb.Simulation(n, prm, stream)
    sim.set_state(X, V, M)
    nb.nbody_set_timing(sim.h, True)

    def step():
        sim.integrate(SEG)
        return sim.vjp(XB, None, X0B, V0B)

    for _ in range(args.warmup):
        step()
    nb.nbody_kernel_times(sim.h)  # reset the per-kernel sums

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    launches0 = nb.nbody_launch_count()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for k in range(args.steps):
        ev[3 * k].record(stream)
        sim.integrate(SEG)
        ev[3 * k + 1].record(stream)
        sim.vjp(XB, None, X0B, V0B)
        ev[3 * k + 2].record(stream)
    t_end.record(stream)
    barrier()
    launches = nb.nbody_launch_count() - launches0
    clk = clocks.stop()
    total_ms = t_start.elapsed_time(t_end)
    fwd_ms = sum(ev[3 * k].elapsed_time(ev[3 * k + 1]) for k in range(args.steps))
    bwd_ms = sum(ev[3 * k + 1].elapsed_time(ev[3 * k + 2]) for k in range(args.steps))
    kt = nb.nbody_kernel_times(sim.h)
    total_ms, value = aggregate(total_ms, 2.0 * n * n * SEG * args.steps, world)
    ms_per_step = total_ms / args.steps

    peaks = nb.nbody_peaks(stream)
    # roofline of the dominant kernel (FP32 CUDA-core bound, "alu")
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peak_max = sms * FP32_LANES * 2 * 2070e6 / 1e12
    kernels = {}
    eqm = bool(np.all(m == m[0]))
    ffma_meas = peaks.get("fp32x2_fma_tflops") or None
    for name, flops in (("pair", FLOPS_PAIR), ("vjp", FLOPS_VJP)):
        ms, cnt = kt[name]
        if cnt:
            avg_s = ms / cnt / 1e3
            ach = flops * n * n / avg_s / 1e12
            ex = EXEC_FLOPS[(name, eqm)]
            ach_ex = ex * n * n / avg_s / 1e12
            kernels[name] = {"launches": cnt, "total_ms": ms, "avg_ms": avg_s * 1e3,
                             "flops_per_interaction": flops,
                             "interactions_per_s": n * n / avg_s,
                             "achieved_tflops": ach, "frac_of_peak_at_2070MHz": ach / peak_max,
                             "executed_flops_per_interaction": ex,
                             "executed_tflops": ach_ex,
                             "frac_executed_of_peak_at_2070MHz": ach_ex / peak_max,
                             "frac_executed_of_measured_ffma":
                                 ach_ex / ffma_meas if ffma_meas else None}
    # O(N) FP64 kernels: algorithmic bytes per particle of an interior launch
    # (update: x, v read and written, S partial slices read, FP32 restage;
    # adjoint: cotangents, tape x, a_pair, v_half, x_prev, m read, cotangents
    # written, S partial slices read, adjoint restage, and the external
    # field's nine adjoint terms computed beside the pair VJP read)
    s_f = nb.nbody_get_pair_shape(sim.h, 0)[3]
    s_v = nb.nbody_get_pair_shape(sim.h, 1)[3]
    bpp = {"update": 48 + 24 * s_f + 48 + 12,
           "adjoint": 48 + 72 + 24 * s_v + 56 + 48 + 32 + 72}
    # field: the FP64 external field of a forward point (x read, field
    # written), on the side stream beside the pair kernel
    bpp["field"] = 48
    hbm = hbm_peak()
    for name in ("update", "adjoint", "field"):
        ms, cnt = kt[name]
        k = {"launches": cnt, "total_ms": ms, "avg_ms": ms / cnt if cnt else None,
             "algorithmic_bytes_per_particle": bpp[name], "bound": "fp64 alu / hbm"}
        if cnt:
            gbs = bpp[name] * n / (ms / cnt / 1e3) / 1e9
            k.update({"achieved_gbs": gbs, "frac_of_hbm": gbs / hbm, "hbm_peak_gbs": hbm})
        kernels[name] = k
    dom = max(("pair", "vjp"), key=lambda k: kt[k][0])
    d = kernels[dom]
    sm_mhz = clk["sm_mhz"] if clk else None
    roofline = {"bound": "alu", "kernel": dom, "achieved": d["achieved_tflops"],
                "peak": peak_max, "unit": "TFLOP/s",
                "frac": d["achieved_tflops"] / peak_max,
                "flops_per_interaction": d["flops_per_interaction"],
                "executed_flops_per_interaction": d["executed_flops_per_interaction"],
                "frac_executed": d["frac_executed_of_peak_at_2070MHz"],
                "peak_measured_ffma": ffma_meas,
                "frac_executed_of_measured_ffma": d["frac_executed_of_measured_ffma"],
                "traffic": traffic_record(dom),
                "peak_basis": "%d SMs x %d FP32 lanes x 2 flop x 2070 MHz (max SM clock)"
                              % (sms, FP32_LANES),
                "frac_at_measured_clock": (d["achieved_tflops"] / (peak_max * sm_mhz / 2070.0))
                if sm_mhz else None,
                "measured_unit_peaks": peaks}

    # end to end through the C ABI with pinned host buffers
    xh = torch.tensor(x.T.copy()).pin_memory()
    vh = torch.tensor(v.T.copy()).pin_memory()
    mh = torch.tensor(m).pin_memory()
    xbh = torch.tensor(xbar.T.copy()).pin_memory()
    x0h = torch.empty((3, n), dtype=torch.float64).pin_memory()
    v0h = torch.empty((3, n), dtype=torch.float64).pin_memory()
    e2e_steps = max(1, args.steps if args.e2e_steps is None else args.e2e_steps)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.set_state(xh, vh, mh)
        sim.integrate(SEG)
        sim.vjp(xbh, None, x0h, v0h)
    barrier()
    e2e_ms, e2e_value = aggregate((time.perf_counter() - t0) / e2e_steps * 1e3,
                                  2.0 * n * n * SEG, world)
    e2e_s = e2e_ms / 1e3
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": int((3 + 3 + 1 + 3) * n * 8),
           "d2h_bytes_per_step": int((3 + 3) * n * 8 + 4 * 8),
           "steps": e2e_steps, "ms_per_step": e2e_s * 1e3}

    # secondary workloads run after the timed region; a failure of one is
    # recorded in the line (as {"error": ...}) instead of losing the line
    def secondary(fn):
        try:
            return fn()
        except Exception as e:  # noqa: BLE001
            return {"error": "%s: %s" % (type(e).__name__, e)}

    ens = None
    if not args.no_ensemble:
        ens = secondary(lambda: measure_ensemble(dev, props.name))

    def grid_and_bootstrap():
        # the point-cloud grid search at the paper's stage-1 size: 10^4
        # simulations of 1000 particles, 1000 steps, ranked by batched MMD;
        # with --bootstrap also 1000 realisations of the observation scored
        # against every kept grid cloud, then all 1000 refined by 10 batched
        # gradient steps
        from paper_2511_22468_gb300 import gridsearch
        nb_boot = 1000 if args.bootstrap else 0
        g = gridsearch.run(refine_iters=10, device=str(dev), bootstrap=nb_boot,
                           bootstrap_refine=nb_boot, refine_batch=500)
        out = {"workload": "grid_1e4_n1000_steps1000", **g["grid"],
               "grid_points": g["workload"]["grid_points"]}
        b = g.get("bootstrap")
        if b:
            out["bootstrap"] = {"realisations": b["realisations"], "cross_mmd_s": b["time_s"],
                                "cross_kernel_pairs_per_s": b["kernel_pairs_per_s"],
                                "refine_s": b["refine"]["time_s"],
                                "refine_iters": b["refine"]["iters"],
                                "refine_batch": b["refine"]["batch"]}
        return out

    grid = None
    if not args.no_grid:
        grid = secondary(grid_and_bootstrap)

    stream_c1 = None
    if not args.no_stream:
        stream_c1 = secondary(lambda: measure_stream_c1(dev, peak_max))

    def recovery():
        # time to a 5 % error on all four parameters (N = 1e4, 100 Myr,
        # point-cloud loss) for the plain descent, the batched grid stage
        # then descent, the surrogate warm start, and the surrogate's start
        # refined by the grid stage, one observation
        from paper_2511_22468_gb300 import warmstart
        r = warmstart.run(observations=(warmstart.F_OBS,), device=str(dev))
        o = r["observations"][0]
        out = {"workload": "gd1_stream_n10k_100myr_mmd", "err_target": r["workload"]["err_target"],
               "f_obs": o["f_obs"], "surrogate_training": r["surrogate_training"]}
        for k in ("plain", "batched", "surrogate", "surrogate_grid"):
            x = o[k]
            out[k] = {key: x[key] for key in ("reached", "time_to_target_s", "final_err",
                                              "start_err", "iters")}
            for key in ("grid_calls", "grid_s", "theta0_err", "inversion_and_grid_s",
                        "time_incl_data_and_training_s"):
                if key in x:
                    out[k][key] = x[key]
        return out

    rec = None
    if not args.no_recovery:
        rec = secondary(recovery)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ra, rv = 8192, 1024
        step_s, wall = oracle_sample(x, m, C3.G, C3.eps, ra, rv)
        cpu = {"value": 2.0 * n * n * SEG / step_s, "unit": UNIT, "cores": cpu_cores(),
               "kind": "oracle",
               "sample": "oracle pair force on %d and pair VJP on %d sampled rows "
                         "against all N = %d, scaled to one step's %d forward + %d "
                         "recomputed + %d VJP passes" % (ra, rv, n, SEG, SEG - 1, SEG + 1),
               "wall_s": wall}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "state_dtype": "f64",
                "data": "synthetic (seeded Plummer sphere)", "config": config_json(C3),
                "fwd_interactions_per_s": n * n * SEG * args.steps * world / (fwd_ms / 1e3),
                "adjoint_ms_per_step": bwd_ms / args.steps,
                "fwd_ms_per_step": fwd_ms / args.steps,
                "pct_fp32_peak": {k: 100.0 * kernels[k]["frac_of_peak_at_2070MHz"]
                                  for k in ("pair", "vjp") if k in kernels},
                "batched_sims_per_s": ens["sims_per_s"] * world if ens and "sims_per_s" in ens
                else None,
                "ensemble": ens,
                "grid_search": grid,
                "stream_c1": stream_c1,
                "recovery": rec,
                "roofline": roofline, "kernels": kernels, "cpu_baseline": cpu,
                "clocks": clk, "e2e": e2e, "gpu_launches": int(launches),
                "parallelism": "replicas" if world > 1 else "single"}
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.steps < 1 or args.warmup < 0:
        raise SystemExit("--steps must be >= 1")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

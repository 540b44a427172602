"""Small profiling case for ncu captures of the pair kernels.

Runs one short forward + adjoint of a Plummer sphere in the NFW + MN
potential through the C ABI (same kernels and launch-shape rules as the
N = 1e6 workload, at a size whose launches take milliseconds):

    python -m paper_2511_22468_gb300.profile_case [--n 262144] [--steps 2]
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=262144)
    ap.add_argument("--steps", type=int, default=2)
    a = ap.parse_args()
    import torch

    from paper_2511_22468_gb300 import build, nbody as nb
    from paper_2511_22468_gb300.configs import C3
    from paper_2511_22468_gb300.inputs import plummer_sphere
    build.build()
    dev = torch.device("cuda:0")
    x, v, m = plummer_sphere(a.n, C3.seed, C3.G, C3.M, C3.a, center=C3.X0, velocity=C3.V0)
    p = C3.pot
    prm = nb.make_params(C3.G, C3.eps, C3.dt, checkpoint_every=a.steps, ext_flags=3,
                         nfw_M=p.nfw_M, nfw_rs=p.nfw_rs, mn_M=p.mn_M, mn_a=p.mn_a,
                         mn_b=p.mn_b, center=C3.X0, center_vel=C3.V0,
                         center_mode=nb.NBODY_CENTER_GUIDE, tape_mode=nb.NBODY_TAPE_LEAN)
    sim = nb.Simulation(a.n, prm)
    sim.set_state(torch.tensor(x.T.copy(), device=dev), torch.tensor(v.T.copy(), device=dev),
                  torch.tensor(m, device=dev))
    sim.integrate(a.steps)
    xb = torch.tensor(np.random.default_rng(0).normal(size=(3, a.n)), device=dev)
    tb = sim.vjp(xb, None)
    torch.cuda.synchronize()
    print("profile case n=%d steps=%d theta_bar=%s launches=%d"
          % (a.n, a.steps, tb, nb.nbody_launch_count()))
    sim.close()


if __name__ == "__main__":
    main()

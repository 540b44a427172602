"""Workload definitions (sizes, units, physical constants, seeds).

Astrophysical workloads use kpc, Myr and solar masses:
G = 4.30091e-6 kpc (km/s)^2 / Msun with 1 km/s = 1.0227122e-3 kpc/Myr gives
G = 4.49850215e-12 kpc^3 / (Msun Myr^2).  The isolated Plummer workload uses
N-body units G = M = a = 1.

The potential is the NFW halo plus Miyamoto-Nagai disk of MWPotential2014
(paper Sec. 2.2.1); the parameter vector is
Theta = (t_end, M_Plummer, M_NFW, M_MN) (Sec. 2.2.1, Fig. 2).  The NFW mass
is read as the scale mass 4 pi rho_0 r_s^3.
"""
from __future__ import annotations

from dataclasses import dataclass, field

G_KPC_MSUN_MYR = 4.49850215e-12

# present-day progenitor centre of mass of the synthetic GD-1-like stream:
# |X| = 14.0 kpc, V perpendicular to X, inclined 30 degrees, L_z < 0
GD1_X0 = (-8.0, 0.0, 11.5)
GD1_V0 = (0.230 * 0.4105, 0.230 * 0.866, 0.230 * 0.2855)
OBSERVER = (-8.0, 0.0, 0.0)


@dataclass(frozen=True)
class Potential:
    nfw_M: float = 1.0e12
    nfw_rs: float = 16.0
    mn_M: float = 6.8e10
    mn_a: float = 3.0
    mn_b: float = 0.28


@dataclass(frozen=True)
class PlummerC0:
    """Isolated Plummer sphere, N-body units, no external potential."""
    name: str = "plummer_n1024"
    n: int = 1024
    G: float = 1.0
    M: float = 1.0
    a: float = 1.0
    eps: float = 0.01
    dt: float = 1.0e-3
    n_steps: int = 1000
    seed: int = 0


@dataclass(frozen=True)
class StreamC1:
    """GD-1-like stream: Plummer progenitor in NFW + MN, 3 Gyr at 0.5 Myr."""
    name: str = "gd1_stream_n10k"
    n: int = 10_000
    G: float = G_KPC_MSUN_MYR
    M_prog: float = 2.0e4
    a_prog: float = 0.010
    eps: float = 0.001
    t_acc: float = 3000.0
    n_steps: int = 6000
    seed: int = 1
    pot: Potential = field(default_factory=Potential)
    X0: tuple = GD1_X0
    V0: tuple = GD1_V0
    observer: tuple = OBSERVER
    # soft 2-D histogram of (phi1, phi2): 32 x 32 bins on
    # phi1 in [-90, 90] deg and phi2 in [-10, 10] deg
    nb1: int = 32
    nb2: int = 32
    phi1_deg: tuple = (-90.0, 90.0)
    phi2_deg: tuple = (-10.0, 10.0)

    @property
    def theta_true(self):
        return (self.t_acc, self.M_prog, self.pot.nfw_M, self.pot.mn_M)


@dataclass(frozen=True)
class EnsembleC2:
    """64 simulations, N log-uniform in [2048, 32768], +-30% parameters."""
    name: str = "ensemble_64"
    n_sims: int = 64
    n_lo: int = 2048
    n_hi: int = 32768
    width: float = 0.30
    n_steps: int = 2000
    steps_per_t_acc: int = 6000
    seed_sizes: int = 100
    seed_params: int = 101
    seed_ics: int = 100


@dataclass(frozen=True)
class ThroughputC3:
    """N = 1e6 Plummer sphere (1e6 Msun, a = 50 pc) at the stream progenitor's
    present-day phase-space point in the NFW + MN potential; eps = 0.5 pc,
    dt = 0.5 Myr, 100 steps, adjoint checkpoints every 10 steps."""
    name: str = "plummer_n1e6_nfw_mn"
    n: int = 1_000_000
    G: float = G_KPC_MSUN_MYR
    M: float = 1.0e6
    a: float = 0.050
    eps: float = 0.0005
    dt: float = 0.5
    n_steps: int = 100
    checkpoint_every: int = 10
    seed: int = 2
    pot: Potential = field(default_factory=Potential)
    X0: tuple = GD1_X0
    V0: tuple = GD1_V0


@dataclass(frozen=True)
class SurrogateC4:
    """MLP 4 -> 256 -> 256 -> 32x32 (GELU), trained on ensemble simulations."""
    name: str = "surrogate_warm_start"
    n_sims: int = 4096
    n_train: int = 3584
    n_particles: int = 10_000
    width: float = 0.30
    hidden: int = 256
    out: int = 1024
    seed_params: int = 10_000
    threshold: float = 0.05


C0 = PlummerC0()
C1 = StreamC1()
C2 = EnsembleC2()
C3 = ThroughputC3()
C4 = SurrogateC4()

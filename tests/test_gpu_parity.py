"""CUDA path vs the FP64 oracle, through the C ABI (needs a GB300).

Tolerances (stated for the method's FP32 pair sum with FP64 state):
  * acceleration: |a_gpu - a_orc| / (|a_orc| + 1e-3 rms|a_orc|) <= 1e-5 per
    particle;
  * positions after 100 steps: max |dx| / r_scale <= 1e-6 (r_scale = the
    Plummer scale radius);
  * energy and momentum drift within 1e-6 of the oracle's;
  * gradients: relative 1e-4 of the oracle adjoint, particle by particle for
    dL/dx0, dL/dv0 and dL/dm (the acceleration's measure: |g_k - r_k| /
    (|r_k| + 1e-3 rms|r|)), element-wise for every scalar.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import core as orc  # noqa: E402
from paper_2511_22468_gb300 import nbody as nb  # noqa: E402
from paper_2511_22468_gb300.configs import C1, C3  # noqa: E402
from paper_2511_22468_gb300.inputs import plummer_sphere  # noqa: E402
from tolerances import (mass_grad_abs_terms, per_particle_err,  # noqa: E402
                        per_particle_err_fp32_sum)

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22468_gb300 import build
    build.build()
    nb.lib()


def to_gpu(a):
    """(n, 3) numpy -> (3, n) float64 device tensor; (n,) -> (n,)."""
    a = np.asarray(a, np.float64)
    if a.ndim == 2:
        a = a.T
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


def to_np(t):
    a = t.detach().cpu().numpy()
    return a.T.copy() if a.ndim == 2 else a.copy()


def acc_err(a, ref):
    return per_particle_err(a, ref)


# -------------------------------------------------------------- pair force --
@pytest.mark.parametrize("n", [1, 2, 3, 31, 33, 1023, 1025, 4999, 70001])
def test_pair_accel_matches_oracle(n):
    x, v, m = plummer_sphere(max(n, 2), 100 + n, 1.0, 1.0, 1.0)
    x, m = x[:n], m[:n] * np.linspace(0.5, 1.5, n)
    eps = 0.01
    acc = torch.empty((3, n), dtype=torch.float64, device=DEV)
    nb.nbody_pair_accel(to_gpu(x), to_gpu(m), 1.0, eps, (0, 0, 0), acc)
    torch.cuda.synchronize()
    a = to_np(acc)
    rows = None if n <= 5000 else np.random.default_rng(n).choice(n, 512, replace=False)
    ref = orc.pair_accel(x, m, 1.0, eps, rows=rows)
    got = a if rows is None else a[rows]
    if n == 1:
        assert np.all(got == 0.0)
        return
    assert acc_err(got, ref) <= 1e-5


def test_pair_accel_full_size_sampled():
    """The throughput workload (N = 1e6 Plummer sphere, 50 pc, eps 0.5 pc, at
    the stream progenitor's position) in the launch shape the benchmark uses,
    on 384 sampled particles the oracle computes one by one."""
    n = C3.n
    x, v, m = plummer_sphere(n, C3.seed, C3.G, C3.M, C3.a, center=C3.X0)
    acc = torch.empty((3, n), dtype=torch.float64, device=DEV)
    nb.nbody_pair_accel(to_gpu(x), to_gpu(m), C3.G, C3.eps, C3.X0, acc)
    torch.cuda.synchronize()
    rows = np.random.default_rng(7).choice(n, 384, replace=False)
    ref = orc.pair_accel(x, m, C3.G, C3.eps, rows=rows)
    assert acc_err(to_np(acc)[rows], ref) <= 1e-5


def test_full_size_step_and_adjoint_sampled():
    """The benchmark's context at full size (N = 1e6, equal masses: the
    equal-mass force and VJP kernels in their tuned launch shapes, NFW + MN,
    guide origin): one kick-drift-kick step and its reverse sweep with
    xbar = W, vbar = 0, whose closed forms for sampled rows are
      x1 - x0 - dt v0 = (dt^2 / 2) a(x0),
      x0bar - W = (dt^2 / 2) (J_pair + J_ext)(x0)^T W,
    against the oracle on 256 rows (acceleration 1e-5 per particle,
    gradient 1e-4 per particle)."""
    n, dt, pot = C3.n, C3.dt, C3.pot
    x, v, m = plummer_sphere(n, C3.seed, C3.G, C3.M, C3.a, center=C3.X0, velocity=C3.V0)
    sim = _sim(n, C3.G, C3.eps, dt, K=1, ext=3, pot=pot, center=C3.X0, center_vel=C3.V0,
               guide=True)
    sim.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
    xo = torch.empty((3, n), dtype=torch.float64, device=DEV)
    sim.integrate(1, xo)
    W = np.random.default_rng(9).normal(size=(n, 3))
    x0b = torch.empty_like(xo)
    sim.vjp(to_gpu(W), None, x0b, None)
    rows = np.random.default_rng(10).choice(n, 256, replace=False)
    ph = orc.Physics(G=C3.G, eps=C3.eps, ext=orc.NFW | orc.MN, nfw_M=pot.nfw_M,
                     nfw_rs=pot.nfw_rs, mn_M=pot.mn_M, mn_a=pot.mn_a, mn_b=pot.mn_b)
    a_ext = np.array([orc.ext_accel(ph, x[k]) for k in rows])
    a_ref = orc.pair_accel(x, m, C3.G, C3.eps, rows=rows) + a_ext
    got = (to_np(xo)[rows] - x[rows] - dt * v[rows]) / (0.5 * dt * dt)
    assert acc_err(got, a_ref) <= 1e-5
    Jt = orc.pair_vjp(x, m, C3.G, C3.eps, W, rows=rows)
    Jt += np.array([orc.ext_jac(ph, x[k]).T @ W[k] for k in rows])
    gb = (to_np(x0b)[rows] - W[rows]) / (0.5 * dt * dt)
    assert per_particle_err(gb, Jt) <= 1e-4
    sim.close()


# (variant, threads, per thread, chunks (0: automatic), where the chunk sums
# are added (-1: automatic), j-pairs per tile (0: the default))
VJP_SHAPES = [(0, 256, 2, 0, -1, 0), (0, 128, 4, 0, -1, 0), (0, 128, 2, 0, -1, 0),
              (0, 128, 1, 0, -1, 0), (0, 128, 2, 9, 1, 0), (0, 128, 2, 9, 0, 0),
              (0, 64, 2, 0, -1, 0), (0, 64, 2, 17, 1, 0), (0, 128, 2, 19, 1, 128),
              (0, 128, 1, 20, 0, 128), (0, 64, 2, 13, 1, 128)]


@pytest.mark.parametrize("eqm", [False, True])
def test_tile_vjp_and_mass_gradient_sampled(eqm):
    """The tile pair-VJP kernels, general masses (spread over
    [0.5, 1.5] of the mean) and equal masses, with and without the
    per-particle mass gradient, in every supported tile shape (and with the
    chunk sums added by the pair kernel and by the consumer, and with 128-pair
    j-tiles), at N = 70001
    (npad = 70656, a ragged last tile): one kick-drift-kick step and its
    reverse sweep with
    xbar = W, vbar = 0, whose closed forms for sampled rows k are
      x0bar_k - W_k = (dt^2 / 2) ((J_pair + J_ext)(x0)^T W)_k,
      mbar_k       = (dt^2 / 2) sum_i W_i . d a_i / d m_k,
    against the oracle on 256 rows, 1e-4 per particle."""
    n, dt = 70001, 0.5
    x, v, m = plummer_sphere(n, 31, C1.G, 1e5, 0.03, center=C1.X0, velocity=C1.V0)
    if not eqm:
        m = m * np.random.default_rng(32).uniform(0.5, 1.5, n)
    pot = C1.pot
    W = np.random.default_rng(33).normal(size=(n, 3))
    rows = np.random.default_rng(34).choice(n, 256, replace=False)
    ph = orc.Physics(G=C1.G, eps=C1.eps, ext=orc.NFW | orc.MN, nfw_M=pot.nfw_M,
                     nfw_rs=pot.nfw_rs, mn_M=pot.mn_M, mn_a=pot.mn_a, mn_b=pot.mn_b)
    Jt = orc.pair_vjp(x, m, C1.G, C1.eps, W, rows=rows)
    Jt += np.array([orc.ext_jac(ph, x[k]).T @ W[k] for k in rows])
    mref = orc.pair_mass_vjp(x, C1.G, C1.eps, W, rows=rows)
    X, V, M, WG = to_gpu(x), to_gpu(v), to_gpu(m), to_gpu(W)
    for variant, nt, r, chunks, finish, tile in VJP_SHAPES:
        sim = _sim(n, C1.G, C1.eps, dt, K=1, ext=3, pot=pot, center=C1.X0,
                   center_vel=C1.V0, guide=True)
        nb.nbody_set_pair_shape(sim.h, 1, variant, nt, r, chunks)
        if tile:
            nb.nbody_set_pair_tile(sim.h, 1, tile)
            assert nb.nbody_get_pair_tile(sim.h, 1) == tile
        if finish >= 0:
            nb.nbody_set_pair_finish(sim.h, 1, finish)
        sim.set_state(X, V, M)
        sim.integrate(1)
        x0b = torch.empty((3, n), dtype=torch.float64, device=DEV)
        sim.vjp(WG, None, x0b, None)                       # no mass gradient
        gb = (to_np(x0b)[rows] - W[rows]) / (0.5 * dt * dt)
        assert per_particle_err(gb, Jt) <= 1e-4, (variant, nt, r, chunks, finish)
        mb = torch.empty(n, dtype=torch.float64, device=DEV)
        x0b2 = torch.empty_like(x0b)
        sim.vjp(WG, None, x0b2, None, mb)                  # with it
        assert torch.allclose(x0b2, x0b, rtol=1e-12, atol=0.0)
        got = to_np(mb)[rows] / (0.5 * dt * dt)
        assert per_particle_err(got, mref) <= 1e-4, (variant, nt, r, chunks, finish)
        assert tuple(nb.nbody_get_pair_shape(sim.h, 1))[:3] == (variant, nt, r)
        assert sim.status() == 0
        sim.close()


@pytest.mark.parametrize("n", [10000, 70001])
def test_tile_force_shapes_one_step(n):
    """Every tile shape of the pair-force kernel (including the 64-thread
    blocks and the 128-pair j-tiles for small systems), general masses: one
    kick-drift-kick step,
    whose closed form x1 - x0 - dt v0 = (dt^2 / 2) a(x0) gives the
    acceleration, against the oracle (1e-5 per particle; sampled rows for
    the larger n), the chunk sums added by the pair kernel and by the
    consumer (same bits)."""
    x, v, m = plummer_sphere(n, 41, C1.G, 1e5, 0.03, center=C1.X0, velocity=C1.V0)
    m = m * np.random.default_rng(42).uniform(0.5, 1.5, n)
    dt, pot = 0.5, C1.pot
    rows = None if n <= 10000 else np.random.default_rng(43).choice(n, 256, replace=False)
    ph = orc.Physics(G=C1.G, eps=C1.eps, ext=orc.NFW | orc.MN, nfw_M=pot.nfw_M,
                     nfw_rs=pot.nfw_rs, mn_M=pot.mn_M, mn_a=pot.mn_a, mn_b=pot.mn_b)
    sel = np.arange(n) if rows is None else rows
    a_ref = orc.pair_accel(x, m, C1.G, C1.eps, rows=rows)
    a_ref += np.array([orc.ext_accel(ph, x[k]) for k in sel])
    for nt, r, tile in ((128, 4, 0), (128, 8, 0), (256, 4, 0), (256, 2, 0), (128, 2, 0),
                        (128, 1, 0), (64, 2, 0), (64, 4, 0), (128, 4, 128), (128, 2, 128),
                        (128, 1, 128), (64, 2, 128), (64, 4, 128)):
        outs = []
        for fin in (0, 1):
            sim = _sim(n, C1.G, C1.eps, dt, ext=3, pot=pot, center=C1.X0, center_vel=C1.V0,
                       guide=True)
            nb.nbody_set_pair_shape(sim.h, 0, 0, nt, r, 9 if not tile else 19)
            if tile:
                nb.nbody_set_pair_tile(sim.h, 0, tile)
            nb.nbody_set_pair_finish(sim.h, 0, fin)
            sim.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
            xo = torch.empty((3, n), dtype=torch.float64, device=DEV)
            sim.integrate(1, xo)
            assert sim.status() == 0
            sim.close()
            outs.append(xo)
        assert torch.equal(outs[0], outs[1]), (nt, r, tile)
        got = (to_np(outs[0])[sel] - x[sel] - dt * v[sel]) / (0.5 * dt * dt)
        assert acc_err(got, a_ref) <= 1e-5, (nt, r, tile)


# warp-variant shapes (threads, per thread): pair force, pair VJP
WARP_FWD = ((256, 4), (256, 8))
WARP_VJP = ((256, 4), (256, 2))


@pytest.mark.parametrize("n", [3001, 10000])
@pytest.mark.parametrize("eqm", [False, True])
def test_warp_shapes_force_vjp_and_mass_gradient(n, eqm):
    """The split-j warp variants of the pair-force and pair-VJP kernels
    (lanes split the j-range, fixed xor butterfly), each shape with the
    automatic chunk count and with 5 chunks, general masses (spread over
    [0.5, 1.5] of the mean) and equal masses, at N = 3001 (ragged, npad =
    3072) and at the stream workload's N = 10^4: one kick-drift-kick step,
    whose closed form x1 - x0 - dt v0 = (dt^2 / 2) a(x0) gives the
    acceleration (1e-5 per particle), and its reverse sweep with xbar = W,
    vbar = 0, whose closed forms are x0bar - W = (dt^2 / 2) ((J_pair +
    J_ext)(x0)^T W) (1e-4 per particle) and mbar = (dt^2 / 2) sum_i W_i .
    d a_i / d m_k (a sum of terms of either sign whose cancellation reaches
    1e4 at some particles: 1e-4 relative plus the FP32 summation bound
    8 u sum|terms|), against the oracle on every row (N = 3001) or 1024
    sampled rows with the first and last; the pair energy of the forward
    shape against the oracle's (1e-6 relative); repeated runs give the same
    bits."""
    dt, pot = 0.5, C1.pot
    x, v, m = plummer_sphere(n, 51, C1.G, 1e5, 0.03, center=C1.X0, velocity=C1.V0)
    if not eqm:
        m = m * np.random.default_rng(52).uniform(0.5, 1.5, n)
    rows = None if n < 5000 else np.unique(np.concatenate(
        [[0, n - 1], np.random.default_rng(53).choice(n, 1024, replace=False)]))
    sel = np.arange(n) if rows is None else rows
    ph = orc.Physics(G=C1.G, eps=C1.eps, ext=orc.NFW | orc.MN, nfw_M=pot.nfw_M,
                     nfw_rs=pot.nfw_rs, mn_M=pot.mn_M, mn_a=pot.mn_a, mn_b=pot.mn_b)
    a_ref = orc.pair_accel(x, m, C1.G, C1.eps, rows=rows)
    a_ref += np.array([orc.ext_accel(ph, x[k]) for k in sel])
    W = np.random.default_rng(54).normal(size=(n, 3))
    Jt = orc.pair_vjp(x, m, C1.G, C1.eps, W, rows=rows)
    Jt += np.array([orc.ext_jac(ph, x[k]).T @ W[k] for k in sel])
    mref = orc.pair_mass_vjp(x, C1.G, C1.eps, W, rows=rows)
    mabs = mass_grad_abs_terms(x, C1.G, C1.eps, W, rows=rows)
    W_pair = orc.energy(orc.Physics(G=C1.G, eps=C1.eps), x, v, m)["W_pair"]
    X, V, M, WG = to_gpu(x), to_gpu(v), to_gpu(m), to_gpu(W)
    for which, shapes in ((0, WARP_FWD), (1, WARP_VJP)):
        for nt, r in shapes:
            for chunks in (0, 5):
                outs = []
                for rep in range(2):
                    sim = _sim(n, C1.G, C1.eps, dt, K=1, ext=3, pot=pot, center=C1.X0,
                               center_vel=C1.V0, guide=True)
                    nb.nbody_set_pair_shape(sim.h, which, 1, nt, r, chunks)
                    assert tuple(nb.nbody_get_pair_shape(sim.h, which))[:3] == (1, nt, r)
                    sim.set_state(X, V, M)
                    if which == 0 and rep == 0:
                        assert sim.energy()[1] == pytest.approx(W_pair, rel=1e-6), (nt, r)
                    xo = torch.empty((3, n), dtype=torch.float64, device=DEV)
                    sim.integrate(1, xo)
                    x0b = torch.empty_like(xo)
                    mb = torch.empty(n, dtype=torch.float64, device=DEV)
                    sim.vjp(WG, None, x0b, None, mb)
                    assert sim.status() == 0
                    sim.close()
                    outs.append((xo, x0b, mb))
                key = (which, nt, r, chunks)
                for a, b in zip(*outs):
                    assert torch.equal(a, b), key
                xo, x0b, mb = outs[0]
                got = (to_np(xo)[sel] - x[sel] - dt * v[sel]) / (0.5 * dt * dt)
                assert acc_err(got, a_ref) <= 1e-5, key
                gb = (to_np(x0b)[sel] - W[sel]) / (0.5 * dt * dt)
                assert per_particle_err(gb, Jt) <= 1e-4, key
                gm = to_np(mb)[sel] / (0.5 * dt * dt)
                assert per_particle_err_fp32_sum(gm, mref, mabs) <= 1.0, key


# --------------------------------------------------------------- trajectory --
def _sim(n, G, eps, dt, K=0, ext=0, pot=None, center=(0, 0, 0), center_vel=(0, 0, 0),
         guide=False, lean=False):
    kw = {}
    if pot is not None:
        kw = dict(nfw_M=pot.nfw_M, nfw_rs=pot.nfw_rs, mn_M=pot.mn_M, mn_a=pot.mn_a,
                  mn_b=pot.mn_b)
    p = nb.make_params(G, eps, dt, checkpoint_every=K, ext_flags=ext, center=center,
                       center_vel=center_vel,
                       center_mode=nb.NBODY_CENTER_GUIDE if guide else nb.NBODY_CENTER_FIXED,
                       tape_mode=nb.NBODY_TAPE_LEAN if lean else nb.NBODY_TAPE_KEEP_LAST, **kw)
    return nb.Simulation(n, p)


@pytest.mark.parametrize("uneq", [False, True])
def test_plummer_trajectory_energy_momentum(uneq):
    """Isolated Plummer sphere (N = 1024, eps = 0.01, dt = 1e-3): positions
    after 100 steps, energy and momentum drift against the oracle (equal
    masses, and masses spread over [0.5, 1.5] of the mean)."""
    n, eps, dt, steps = 1024, 0.01, 1e-3, 100
    x, v, m = plummer_sphere(n, 0, 1.0, 1.0, 1.0)
    if uneq:
        m = m * np.linspace(0.5, 1.5, n)
    sim = _sim(n, 1.0, eps, dt)
    sim.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
    e0 = sim.energy()
    P0 = np.array(sim.momentum())
    xo = torch.empty((3, n), dtype=torch.float64, device=DEV)
    vo = torch.empty_like(xo)
    sim.integrate(steps, xo, vo)
    e1 = sim.energy()
    P1 = np.array(sim.momentum())
    ph = orc.Physics(G=1.0, eps=eps)
    xr, vr = orc.integrate(ph, x, v, m, dt, steps)
    assert np.abs(to_np(xo) - xr).max() / 1.0 <= 1e-6
    E0o = orc.energy(ph, x, v, m)
    E1o = orc.energy(ph, xr, vr, m)
    assert e0[0] + e0[1] + e0[2] == pytest.approx(E0o["E"], rel=1e-6)
    dE_gpu = (e1[0] + e1[1] + e1[2]) / (e0[0] + e0[1] + e0[2]) - 1
    dE_orc = E1o["E"] / E0o["E"] - 1
    assert abs(dE_gpu - dE_orc) <= 1e-6
    sig = np.sqrt(np.mean(np.sum(v * v, axis=1)))
    assert np.abs(P1 - P0).max() / (m.sum() * sig) <= 1e-6
    assert sim.status() == 0


def test_step_calls_equal_one_integrate_call():
    """Two 25-step calls continue the same trajectory as one 50-step call
    (cached first-same-as-last acceleration), to rounding of the split kick."""
    n = 512
    x, v, m = plummer_sphere(n, 4, 1.0, 1.0, 1.0)
    a = _sim(n, 1.0, 0.02, 2e-3)
    b = _sim(n, 1.0, 0.02, 2e-3)
    for s in (a, b):
        s.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
    a.step(50)
    b.step(25)
    b.step(25)
    xa = torch.empty((3, n), dtype=torch.float64, device=DEV)
    xb = torch.empty_like(xa)
    a.get_state(xa)
    b.get_state(xb)
    assert (xa - xb).abs().max().item() <= 1e-12


def test_external_potential_stream_segment():
    """Stream progenitor (N = 2048, 10 pc, eps = 1 pc) on its orbit in
    NFW + MN, 100 steps of 0.5 Myr, guided recentring: positions against the
    oracle."""
    n, steps = 2048, 100
    x, v, m = plummer_sphere(n, 3, C1.G, C1.M_prog, C1.a_prog, center=C1.X0, velocity=C1.V0)
    p = C1.pot
    sim = _sim(n, C1.G, C1.eps, 0.5, ext=3, pot=p, center=C1.X0, center_vel=C1.V0, guide=True)
    sim.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
    xo = torch.empty((3, n), dtype=torch.float64, device=DEV)
    sim.integrate(steps, xo)
    ph = orc.Physics(G=C1.G, eps=C1.eps, ext=orc.NFW | orc.MN, nfw_M=p.nfw_M,
                     nfw_rs=p.nfw_rs, mn_M=p.mn_M, mn_a=p.mn_a, mn_b=p.mn_b)
    xr, vr = orc.integrate(ph, x, v, m, 0.5, steps)
    d = np.linalg.norm(to_np(xo) - xr, axis=1)
    # positions relative error per particle, and the internal structure:
    # rms displacement error against the 10 pc Plummer scale (the worst
    # particle sits near 1e-6 a after ~15 dynamical times: FP32 rounding of
    # x - c, 2e-9 kpc at 20 pc, amplified by the cluster's chaos)
    assert np.max(d / np.linalg.norm(xr, axis=1)) <= 1e-6
    assert np.sqrt(np.mean(d * d)) / C1.a_prog <= 1e-6
    assert np.max(d) / C1.a_prog <= 1e-5


def test_bitwise_reproducible():
    n = 3000
    x, v, m = plummer_sphere(n, 8, 1.0, 1.0, 1.0)
    outs = []
    for _ in range(2):
        s = _sim(n, 1.0, 0.01, 1e-3)
        s.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
        o = torch.empty((3, n), dtype=torch.float64, device=DEV)
        s.integrate(30, o)
        outs.append(o)
    assert torch.equal(outs[0], outs[1])


# ------------------------------------------------------------------ adjoint --
@pytest.mark.parametrize("K,lean,ext,uneq", [(7, False, 0, False), (10, True, 0, False),
                                             (50, False, 3, False), (4, True, 3, False),
                                             (7, False, 0, True), (9, True, 3, True)])
def test_adjoint_matches_oracle(K, lean, ext, uneq):
    """Discrete adjoint against the oracle's: dL/dx0, dL/dv0, dL/dm particle
    by particle, dL/ddt, the mass scale, dL/dM_NFW, dL/dM_MN; ragged last
    segments (50 = 7*7 + 1); equal masses (the kernels that leave the mass
    out) and unequal ones.  The cluster on its orbit takes steps of 0.1 Myr:
    the 50 steps span 1.5 dynamical times (3.3 Myr), where the gradient of
    each particle is well conditioned (longer runs: the envelope test
    below)."""
    n, steps = 256, 50
    if ext:
        x, v, m = plummer_sphere(n, 12, C1.G, C1.M_prog, C1.a_prog, center=C1.X0,
                                 velocity=C1.V0)
        G, eps, dt, pot = C1.G, C1.eps, 0.1, C1.pot
    else:
        x, v, m = plummer_sphere(n, 12, 1.0, 1.0, 1.0)
        G, eps, dt, pot = 1.0, 0.05, 2e-3, None
    if uneq:
        m = m * np.linspace(0.5, 1.5, n)
    sim = _sim(n, G, eps, dt, K=K, ext=ext, pot=pot, center=x.mean(axis=0),
               center_vel=v.mean(axis=0), guide=bool(ext), lean=lean)
    sim.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
    sim.integrate(steps)
    rng = np.random.default_rng(K)
    wx = rng.normal(size=(n, 3))
    wv = rng.normal(size=(n, 3))
    x0b = torch.empty((3, n), dtype=torch.float64, device=DEV)
    v0b = torch.empty_like(x0b)
    tb = sim.vjp(to_gpu(wx), to_gpu(wv), x0b, v0b)
    if ext:
        ph = orc.Physics(G=G, eps=eps, ext=orc.NFW | orc.MN, nfw_M=pot.nfw_M,
                         nfw_rs=pot.nfw_rs, mn_M=pot.mn_M, mn_a=pot.mn_a, mn_b=pot.mn_b)
    else:
        ph = orc.Physics(G=G, eps=eps)
    r = orc.vjp(ph, x, v, m, dt, steps, wx, wv)
    for got, ref in ((to_np(x0b), r["x0bar"]), (to_np(v0b), r["v0bar"])):
        assert per_particle_err(got, ref) <= 1e-4
    assert tb[0] == pytest.approx(r["dt_bar"], rel=1e-4)
    assert tb[1] == pytest.approx(np.dot(m, r["mbar"]), rel=1e-4)
    if ext:
        assert tb[2] == pytest.approx(r["nfw_M_bar"], rel=1e-4)
        assert tb[3] == pytest.approx(r["mn_M_bar"], rel=1e-4)
        pg = sim.potential_grad()
        assert pg[:5] == pytest.approx([r["nfw_M_bar"], r["nfw_rs_bar"], r["mn_M_bar"],
                                        r["mn_a_bar"], r["mn_b_bar"]], rel=1e-4)
        assert pg[5] == 0.0
    # a second reverse sweep over the same tape gives the same result
    tb2 = sim.vjp(to_gpu(wx), to_gpu(wv), x0b2 := torch.empty_like(x0b), None)
    assert torch.equal(x0b, x0b2) and tb2 == tb
    # per-particle mass gradients: against the oracle, the identity
    # sum_j m_j dL/dm_j = theta_bar[1], no change to the other outputs, and
    # reproducible from sweep to sweep
    mb = torch.empty(n, dtype=torch.float64, device=DEV)
    tb3 = sim.vjp(to_gpu(wx), to_gpu(wv), x0b3 := torch.empty_like(x0b), None, mb)
    got = to_np(mb)
    assert per_particle_err(got, r["mbar"]) <= 1e-4
    assert float(np.dot(m, got)) == pytest.approx(tb3[1], rel=1e-5)
    assert torch.allclose(x0b3, x0b, rtol=1e-12, atol=0.0)
    assert tb3 == pytest.approx(tb, rel=1e-12)
    mb2 = torch.empty_like(mb)
    sim.vjp(to_gpu(wx), to_gpu(wv), None, None, mb2)
    assert torch.equal(mb, mb2)


def test_adjoint_chaotic_horizon_within_oracle_envelope():
    """Over 7.5 dynamical times (50 steps of 0.5 Myr) the cluster's chaos
    amplifies a perturbation by ~e^7.5, so no FP32 force sum can follow the
    FP64 oracle's trajectory to 1e-4 per particle: the oracle itself, run
    from positions perturbed by 6e-8 relative (the FP32 rounding of x - c),
    differs from its own gradients by ~3e-4 per particle in dL/dm.  Bound:
    per particle, the GPU stays within 4x the larger of two such envelopes
    (and 1e-4); norm-wise and for every scalar, 1e-4 relative."""
    n, steps, dt, pot = 256, 50, 0.5, C1.pot
    x, v, m = plummer_sphere(n, 12, C1.G, C1.M_prog, C1.a_prog, center=C1.X0, velocity=C1.V0)
    sim = _sim(n, C1.G, C1.eps, dt, K=9, ext=3, pot=pot, center=x.mean(axis=0),
               center_vel=v.mean(axis=0), guide=True)
    sim.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
    sim.integrate(steps)
    rng = np.random.default_rng(50)
    wx, wv = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    x0b = torch.empty((3, n), dtype=torch.float64, device=DEV)
    v0b = torch.empty_like(x0b)
    mb = torch.empty(n, dtype=torch.float64, device=DEV)
    tb = sim.vjp(to_gpu(wx), to_gpu(wv), x0b, v0b, mb)
    ph = orc.Physics(G=C1.G, eps=C1.eps, ext=orc.NFW | orc.MN, nfw_M=pot.nfw_M,
                     nfw_rs=pot.nfw_rs, mn_M=pot.mn_M, mn_a=pot.mn_a, mn_b=pot.mn_b)
    r = orc.vjp(ph, x, v, m, dt, steps, wx, wv)
    c = x.mean(axis=0)
    env = {"x0bar": 0.0, "v0bar": 0.0, "mbar": 0.0}
    for seed in (1, 2):
        xp = c + (x - c) * (1.0 + 6e-8 * np.random.default_rng(seed).standard_normal(x.shape))
        rp = orc.vjp(ph, xp, v, m, dt, steps, wx, wv)
        for k in env:
            env[k] = max(env[k], per_particle_err(rp[k], r[k]))
    for k, got in (("x0bar", to_np(x0b)), ("v0bar", to_np(v0b)), ("mbar", to_np(mb))):
        assert per_particle_err(got, r[k]) <= max(1e-4, 4.0 * env[k]), (k, env[k])
        assert np.linalg.norm(got - r[k]) <= 1e-4 * np.linalg.norm(r[k]), k
    assert tb[0] == pytest.approx(r["dt_bar"], rel=1e-4)
    assert tb[1] == pytest.approx(np.dot(m, r["mbar"]), rel=1e-4)
    assert tb[2] == pytest.approx(r["nfw_M_bar"], rel=1e-4)
    assert tb[3] == pytest.approx(r["mn_M_bar"], rel=1e-4)
    sim.close()


# ------------------------------------------------------------ error paths --
def test_errors_are_reported():
    p = nb.make_params(1.0, 0.0, 1e-3)
    with pytest.raises(nb.NBodyError) as e:
        nb.Simulation(10, p)
    assert e.value.code == nb.NBODY_EINVAL
    sim = _sim(10, 1.0, 0.1, 1e-3)
    x, v, m = plummer_sphere(10, 1, 1.0, 1.0, 1.0)
    sim.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
    sim.integrate(3)
    with pytest.raises(nb.NBodyError) as e:  # no tape (checkpoint_every = 0)
        sim.vjp(to_gpu(x), None)
    assert e.value.code == nb.NBODY_ESTATE
    with pytest.raises(nb.NBodyError) as e:  # no gradient computed yet
        sim.potential_grad()
    assert e.value.code == nb.NBODY_ESTATE
    with pytest.raises(nb.NBodyError):
        sim.integrate(0)
    # a non-finite input is caught by the update kernel and reported
    x[3, 1] = np.nan
    sim.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
    sim.step(2)
    assert sim.status() == nb.NBODY_ENAN


# ------------------------------------------------ resume, graphs, autotune --
def test_resume_from_saved_state():
    """Checkpoint / resume: a run continued in a new context from the saved
    state matches one uninterrupted run (to the rounding of the split kick)."""
    n = 2048
    x, v, m = plummer_sphere(n, 21, 1.0, 1.0, 1.0)
    one = _sim(n, 1.0, 0.01, 1e-3)
    one.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
    xa = torch.empty((3, n), dtype=torch.float64, device=DEV)
    one.integrate(50, xa)
    first = _sim(n, 1.0, 0.01, 1e-3)
    first.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
    xs = torch.empty((3, n), dtype=torch.float64, device=DEV)
    vs = torch.empty_like(xs)
    first.integrate(30, xs, vs)
    saved = (xs.cpu().numpy().copy(), vs.cpu().numpy().copy())   # to host and back
    second = _sim(n, 1.0, 0.01, 1e-3)
    second.set_state(torch.tensor(saved[0], device=DEV), torch.tensor(saved[1], device=DEV),
                     to_gpu(m))
    xb = torch.empty_like(xs)
    second.integrate(20, xb)
    assert (xa - xb).abs().max().item() <= 1e-12


def test_graph_replay_equals_eager_launches():
    """Small systems replay the captured step loop and reverse sweep; event
    timing forces eager launches.  Both give the same bits."""
    n = 3000
    x, v, m = plummer_sphere(n, 22, 1.0, 1.0, 1.0)
    xb = torch.tensor(np.random.default_rng(1).normal(size=(3, n)), device=DEV)
    outs = []
    for eager in (False, True):
        s = _sim(n, 1.0, 0.01, 1e-3, K=6)
        nb.nbody_set_timing(s.h, eager)
        s.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
        xo = torch.empty((3, n), dtype=torch.float64, device=DEV)
        s.integrate(25, xo)
        g = torch.empty_like(xo)
        tb = s.vjp(xb, None, g, None)
        s.integrate(25, xo)   # second call: replay of the cached graph
        outs.append((xo, g, tb))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


@pytest.mark.parametrize("steps,K,lean,fin", [(25, 6, False, 1), (25, 6, True, 0),
                                               (3, 1, False, 1), (14, 7, True, 1)])
def test_overlapped_reverse_sweep_equals_serial(steps, K, lean, fin):
    """Small systems recompute the segment before the one being swept back
    on a second stream, into a second segment buffer with its own pair
    scratch; event timing keeps the serial order.  Both give the same bits
    for dL/dx0, dL/dv0, dL/dm and the parameter gradient (external field,
    unequal masses, an even and odd number of segments, lean and kept last
    segment, chunk sums in the kernel or by the consumer), and a second
    sweep over the same tape repeats the first."""
    n = 3000
    x, v, m = plummer_sphere(n, 26, C1.G, C1.M_prog, C1.a_prog, center=C1.X0, velocity=C1.V0)
    m = m * np.random.default_rng(7).uniform(0.5, 1.5, n)
    xb = torch.tensor(np.random.default_rng(8).normal(size=(3, n)), device=DEV)
    vb = torch.tensor(np.random.default_rng(9).normal(size=(3, n)), device=DEV)
    outs = []
    for serial in (False, True):
        s = _sim(n, C1.G, C1.eps, 0.5, K=K, ext=3, pot=C1.pot, center=x.mean(axis=0),
                 center_vel=v.mean(axis=0), guide=True, lean=lean)
        nb.nbody_set_timing(s.h, serial)
        for vjp in (0, 1):
            nb.nbody_set_pair_shape(s.h, vjp, 0, 128, 1, 9)
            nb.nbody_set_pair_finish(s.h, vjp, fin)
        s.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
        xo = torch.empty((3, n), dtype=torch.float64, device=DEV)
        s.integrate(steps, xo)
        got = []
        for _ in range(2):
            g, gv = torch.empty_like(xo), torch.empty_like(xo)
            gm = torch.empty(n, dtype=torch.float64, device=DEV)
            tb = s.vjp(xb, vb, g, gv, gm)
            got.append((g, gv, gm, list(tb), list(s.potential_grad())))
        for a, b in zip(got[0][:3], got[1][:3]):
            assert torch.equal(a, b)
        assert got[0][3:] == got[1][3:]
        outs.append(got[0])
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert torch.equal(a, b)
    assert outs[0][3:] == outs[1][3:]


@pytest.mark.parametrize("ext,uneq", [(0, False), (3, True)])
def test_chunk_sums_in_kernel_equal_sums_by_consumer(ext, uneq):
    """The chunk sums of a split pair kernel added by its last-finishing
    block or by the update / adjoint kernel give the same bits (same slices,
    same ascending order): trajectory, dL/dx0, dL/dv0, dL/dm and the
    potential-parameter gradient."""
    n = 5000
    if ext:
        x, v, m = plummer_sphere(n, 24, C1.G, C1.M_prog, C1.a_prog, center=C1.X0,
                                 velocity=C1.V0)
        G, eps, dt, pot = C1.G, C1.eps, 0.5, C1.pot
    else:
        x, v, m = plummer_sphere(n, 24, 1.0, 1.0, 1.0)
        G, eps, dt, pot = 1.0, 0.01, 1e-3, None
    if uneq:
        m = m * np.random.default_rng(3).uniform(0.5, 1.5, n)
    xb = torch.tensor(np.random.default_rng(4).normal(size=(3, n)), device=DEV)
    vb = torch.tensor(np.random.default_rng(5).normal(size=(3, n)), device=DEV)
    outs = []
    for mode in (0, 1):
        s = _sim(n, G, eps, dt, K=4, ext=ext, pot=pot, center=x.mean(axis=0),
                 center_vel=v.mean(axis=0), guide=bool(ext))
        for vjp in (0, 1):
            nb.nbody_set_pair_shape(s.h, vjp, 0, 128, 1, 9)
            nb.nbody_set_pair_finish(s.h, vjp, mode)
        s.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
        xo = torch.empty((3, n), dtype=torch.float64, device=DEV)
        vo = torch.empty_like(xo)
        s.integrate(13, xo, vo)
        g, gv = torch.empty_like(xo), torch.empty_like(xo)
        gm = torch.empty(n, dtype=torch.float64, device=DEV)
        tb = s.vjp(xb, vb, g, gv, gm)
        pg = s.potential_grad() if ext else None
        assert s.status() == 0
        outs.append((xo, vo, g, gv, gm, tb, pg))
        s.close()
    a, b = outs
    for k in range(5):
        assert torch.equal(a[k], b[k]), k
    assert a[5] == b[5]
    if ext:
        assert np.array_equal(np.asarray(a[6]), np.asarray(b[6]))


def test_autotuned_shapes_match_oracle():
    n = 5000
    x, v, m = plummer_sphere(n, 23, 1.0, 1.0, 1.0)
    s = _sim(n, 1.0, 0.01, 1e-3, K=5)
    s.set_state(to_gpu(x), to_gpu(v), to_gpu(m))
    f, b = nb.nbody_autotune_pair(s.h, 2)
    assert nb.nbody_get_pair_shape(s.h, 0) == f and nb.nbody_get_pair_shape(s.h, 1) == b
    xo = torch.empty((3, n), dtype=torch.float64, device=DEV)
    s.integrate(5, xo)
    xr, _ = orc.integrate(orc.Physics(G=1.0, eps=0.01), x, v, m, 1e-3, 5)
    assert np.abs(to_np(xo) - xr).max() <= 1e-6
    lam = np.random.default_rng(2).normal(size=(n, 3))
    tb = s.vjp(to_gpu(lam), None, g := torch.empty_like(xo), None)
    r = orc.vjp(orc.Physics(G=1.0, eps=0.01), x, v, m, 1e-3, 5, lam, np.zeros_like(lam),
                want_mbar=False)
    assert per_particle_err(to_np(g), r["x0bar"]) <= 1e-4


def test_autograd_simulate_matches_oracle():
    """nb.simulate as a torch autograd function: gradients for x0, v0, the
    per-particle masses and (dt, M_NFW, M_MN) against the oracle adjoint."""
    n, steps = 200, 40
    x, v, m = plummer_sphere(n, 21, C1.G, C1.M_prog, C1.a_prog, center=C1.X0, velocity=C1.V0)
    m = m * np.linspace(0.8, 1.2, n)
    pot = C1.pot
    sim = _sim(n, C1.G, C1.eps, 0.5, K=8, ext=3, pot=pot, center=x.mean(axis=0),
               center_vel=v.mean(axis=0), guide=True, lean=False)
    X0 = to_gpu(x).requires_grad_()
    V0 = to_gpu(v).requires_grad_()
    M = to_gpu(m).requires_grad_()
    th = torch.tensor([0.5, pot.nfw_M, pot.nfw_rs, pot.mn_M, pot.mn_a, pot.mn_b],
                      dtype=torch.float64, requires_grad=True)
    rng = np.random.default_rng(3)
    wx, wv = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    xT, vT = nb.simulate(sim, X0, V0, M, steps, th)
    loss = (xT * to_gpu(wx)).sum() + (vT * to_gpu(wv)).sum()
    loss.backward()
    ph = orc.Physics(G=C1.G, eps=C1.eps, ext=orc.NFW | orc.MN, nfw_M=pot.nfw_M,
                     nfw_rs=pot.nfw_rs, mn_M=pot.mn_M, mn_a=pot.mn_a, mn_b=pot.mn_b)
    r = orc.vjp(ph, x, v, m, 0.5, steps, wx, wv)
    for got, ref in ((to_np(X0.grad), r["x0bar"]), (to_np(V0.grad), r["v0bar"]),
                     (to_np(M.grad), r["mbar"])):
        assert per_particle_err(got, ref) <= 1e-4
    ref_th = [r["dt_bar"], r["nfw_M_bar"], r["nfw_rs_bar"], r["mn_M_bar"], r["mn_a_bar"],
              r["mn_b_bar"]]
    assert th.grad.tolist() == pytest.approx(ref_th, rel=1e-4)
    sim.close()


def test_ext_accel_matches_oracle():
    """The FP64 external field (Newton-Raphson reciprocal square roots in the
    kernel) against the oracle's correctly rounded expressions, from deep
    inside the NFW series branch (r < 1e-4 r_s) to 200 kpc, on and off the
    disk plane.  Bound per point: 1e-13 of |a| plus the conditioning of the
    NFW difference ln(1+u)/r^3 - 1/(r^2 (r+r_s)), whose terms exceed the
    result by about 4/u (u = r/r_s): 2e-15 * 4/u of |a|."""
    rng = np.random.default_rng(8)
    r = np.concatenate([10 ** rng.uniform(-7, -2.5, 300), 10 ** rng.uniform(-2.5, 2.3, 700)])
    u = rng.normal(size=(1000, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    x = r[:, None] * u
    x[::10, 2] = 0.0                      # points in the disk plane
    pot = C1.pot
    for mn_b in (pot.mn_b, 0.0):
        p = nb.make_params(C1.G, C1.eps, 0.5, ext_flags=3, nfw_M=pot.nfw_M, nfw_rs=pot.nfw_rs,
                           mn_M=pot.mn_M, mn_a=pot.mn_a, mn_b=mn_b)
        acc = torch.empty((3, len(x)), dtype=torch.float64, device=DEV)
        nb.nbody_ext_accel(p, to_gpu(x), acc)
        got = to_np(acc)
        ph = orc.Physics(G=C1.G, ext=orc.NFW | orc.MN, nfw_M=pot.nfw_M, nfw_rs=pot.nfw_rs,
                         mn_M=pot.mn_M, mn_a=pot.mn_a, mn_b=mn_b)
        ref = np.array([orc.ext_accel(ph, xi) for xi in x])
        ok = np.all(np.isfinite(ref), axis=1)   # the thin disk's oracle is 0/0 at z = 0
        assert np.all(np.isfinite(got))
        err = np.linalg.norm(got[ok] - ref[ok], axis=1) / np.linalg.norm(ref[ok], axis=1)
        bound = 1e-13 + 2e-15 * 4.0 * pot.nfw_rs / r[ok]
        assert np.all(err <= bound), (err / bound).max()
        if mn_b == 0.0:
            assert np.all(got[~ok][:, 2] == 0.0) and (~ok).sum() >= 50


def test_bulge_field_orbit_and_adjoint_match_oracle():
    """MWPotential2014 with its bulge (incomplete gamma functions by series
    and continued fraction on the GPU, quadrature of the density in the
    oracle): the field from 10 pc to 100 kpc, then a cluster orbiting inside
    the bulge: energy, positions after 40 steps, and the adjoint including
    dL/dM_bulge."""
    pot = C1.pot
    kw = dict(nfw_M=pot.nfw_M, nfw_rs=pot.nfw_rs, mn_M=pot.mn_M, mn_a=pot.mn_a, mn_b=pot.mn_b,
              bulge_M=5e9, bulge_alpha=1.8, bulge_rc=1.9)
    ph = orc.Physics(G=C1.G, eps=1e-3, ext=orc.NFW | orc.MN | orc.BULGE, **kw)
    rng = np.random.default_rng(12)
    r = 10 ** rng.uniform(-2, 2, 400)
    u = rng.normal(size=(400, 3))
    x = r[:, None] * u / np.linalg.norm(u, axis=1)[:, None]
    p = nb.make_params(C1.G, 1e-3, 0.5, ext_flags=7, **kw)
    acc = torch.empty((3, len(x)), dtype=torch.float64, device=DEV)
    nb.nbody_ext_accel(p, to_gpu(x), acc)
    ref = np.array([orc.ext_accel(ph, xi) for xi in x])
    err = np.linalg.norm(to_np(acc) - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= 1e-12 + 8e-15 * pot.nfw_rs / r), err.max()

    n, steps, dt = 64, 40, 0.5
    # a light cluster (1e3 M_sun over 50 pc): the gradient is carried by the
    # field's Jacobian, not by the self-gravity's chaos
    xc, vc, m = plummer_sphere(n, 14, C1.G, 1e3, 0.05, center=(2.0, 0.5, 0.3),
                               velocity=(0.0, 0.2, 0.03))
    sim = _sim(n, C1.G, 1e-3, dt, K=10, ext=7, pot=None, center=xc.mean(axis=0),
               center_vel=vc.mean(axis=0), guide=True)
    prm = sim.params
    prm.nfw_M, prm.nfw_rs, prm.mn_M, prm.mn_a, prm.mn_b = (pot.nfw_M, pot.nfw_rs, pot.mn_M,
                                                         pot.mn_a, pot.mn_b)
    prm.bulge_M, prm.bulge_alpha, prm.bulge_rc = 5e9, 1.8, 1.9
    sim.set_params(prm)
    sim.set_state(to_gpu(xc), to_gpu(vc), to_gpu(m))
    e0 = sim.energy()
    E0 = orc.energy(ph, xc, vc, m)
    assert e0[2] == pytest.approx(E0["W_ext"], rel=1e-12)
    xo = torch.empty((3, n), dtype=torch.float64, device=DEV)
    sim.integrate(steps, xo)
    xr, _ = orc.integrate(ph, xc, vc, m, dt, steps)
    d = np.linalg.norm(to_np(xo) - xr, axis=1)
    assert np.max(d / np.linalg.norm(xr, axis=1)) <= 1e-6
    wx, wv = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    x0b = torch.empty((3, n), dtype=torch.float64, device=DEV)
    tb = sim.vjp(to_gpu(wx), to_gpu(wv), x0b, None)
    rr = orc.vjp(ph, xc, vc, m, dt, steps, wx, wv, want_mbar=False)
    assert per_particle_err(to_np(x0b), rr["x0bar"]) <= 1e-4
    assert tb[0] == pytest.approx(rr["dt_bar"], rel=1e-4)
    pg = sim.potential_grad()
    assert pg == pytest.approx([rr["nfw_M_bar"], rr["nfw_rs_bar"], rr["mn_M_bar"],
                                rr["mn_a_bar"], rr["mn_b_bar"], rr["bulge_M_bar"]], rel=1e-4)
    sim.close()

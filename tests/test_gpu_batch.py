"""Batched ensemble (uneven N, per-simulation parameters, one persistent
pair launch per step, graph-captured step loop) against the oracle and the
single-system path (needs a GB300)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import core as orc  # noqa: E402
from paper_2511_22468_gb300 import nbody as nb  # noqa: E402
from paper_2511_22468_gb300.configs import C1  # noqa: E402
from paper_2511_22468_gb300.inputs import plummer_sphere  # noqa: E402
from tolerances import per_particle_err  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22468_gb300 import build
    build.build()
    nb.lib()


def _members():
    """Three simulations of uneven size: an isolated Plummer sphere in N-body
    units and two stream progenitors on their orbit with different masses,
    potentials and steps."""
    pot = C1.pot
    sims = []
    x, v, m = plummer_sphere(300, 31, 1.0, 1.0, 1.0)
    sims.append((x, v, m, nb.make_params(1.0, 0.02, 2e-3),
                 orc.Physics(G=1.0, eps=0.02)))
    for k, (n, f) in enumerate(((1500, 0.8), (2600, 1.25))):
        x, v, m = plummer_sphere(n, 40 + k, C1.G, C1.M_prog * f, C1.a_prog,
                                 center=C1.X0, velocity=C1.V0)
        dt = 0.5 * f
        p = nb.make_params(C1.G, C1.eps, dt, ext_flags=3, nfw_M=pot.nfw_M * f,
                           nfw_rs=pot.nfw_rs, mn_M=pot.mn_M / f, mn_a=pot.mn_a,
                           mn_b=pot.mn_b, center=C1.X0, center_vel=C1.V0,
                           center_mode=nb.NBODY_CENTER_GUIDE)
        ph = orc.Physics(G=C1.G, eps=C1.eps, ext=orc.NFW | orc.MN, nfw_M=pot.nfw_M * f,
                         nfw_rs=pot.nfw_rs, mn_M=pot.mn_M / f, mn_a=pot.mn_a, mn_b=pot.mn_b)
        sims.append((x, v, m, p, ph))
    return sims


def assert_positions_close(got, ref, ph):
    """Isolated sphere (N-body units): max |dx| <= 1e-6 a.  Sphere on its
    Galactic orbit: per-particle relative error <= 1e-6 and rms <= 1e-6 a
    (the worst particle sits near 1e-6 a: FP32 rounding of x - c amplified
    by the cluster's chaos)."""
    d = np.linalg.norm(got - ref, axis=1)
    if ph.ext == 0:
        assert d.max() <= 1e-6
    else:
        assert np.max(d / np.linalg.norm(ref, axis=1)) <= 1e-6
        assert np.sqrt(np.mean(d * d)) / C1.a_prog <= 1e-6


def _pack(sims):
    offs = np.cumsum([0] + [s[0].shape[0] for s in sims])
    X = np.concatenate([s[0] for s in sims]).T.copy()
    V = np.concatenate([s[1] for s in sims]).T.copy()
    M = np.concatenate([s[2] for s in sims]).copy()
    return offs, torch.tensor(X, device=DEV), torch.tensor(V, device=DEV), torch.tensor(M, device=DEV)


def _run_batch(sims, steps, tuning=None, calls=1):
    offs, X, V, M = _pack(sims)
    h = nb.nbody_create_batch(offs, [s[3] for s in sims])
    try:
        if tuning is not None:
            nb.nbody_set_tuning(h, tuning)
        nb.nbody_set_state(h, X, V, M)
        for _ in range(calls):
            nb.nbody_integrate(h, steps // calls)
        xo = torch.empty_like(X)
        nb.nbody_get_state(h, xo, None)
        assert nb.nbody_get_status(h) == 0
    finally:
        nb.nbody_destroy(h)
    out = xo.cpu().numpy().T
    return [out[offs[k]:offs[k + 1]] for k in range(len(sims))]


@pytest.mark.parametrize("tuning", range(nb.NBODY_NTUNE))
def test_batch_members_match_oracle(tuning):
    sims = _members()
    steps = 40
    got = _run_batch(sims, steps, tuning=tuning)
    for (x, v, m, p, ph), xb in zip(sims, got):
        xr, _ = orc.integrate(ph, x, v, m, p.dt, steps)
        assert_positions_close(xb, xr, ph)


def test_batch_equals_single_runs_and_is_reproducible():
    sims = _members()
    a = _run_batch(sims, 30)
    b = _run_batch(sims, 30)
    for xa, xb in zip(a, b):
        assert np.array_equal(xa, xb)
    for (x, v, m, p, ph), xa in zip(sims, a):
        sim = nb.Simulation(x.shape[0], p)
        sim.set_state(torch.tensor(x.T.copy(), device=DEV), torch.tensor(v.T.copy(), device=DEV),
                      torch.tensor(m, device=DEV))
        xo = torch.empty((3, x.shape[0]), dtype=torch.float64, device=DEV)
        sim.integrate(30, xo)
        assert_positions_close(xo.cpu().numpy().T, xa, ph)
        sim.close()


def test_batch_graph_replay_continues_the_run():
    sims = _members()
    one = _run_batch(sims, 40, calls=1)
    two = _run_batch(sims, 40, calls=2)   # the captured graph is replayed
    for xa, xb, s in zip(one, two, sims):
        scale = 1.0 if s[4].ext == 0 else C1.a_prog
        assert np.abs(xa - xb).max() / scale <= 1e-9


def test_autotune_selects_a_candidate():
    sims = _members()
    offs, X, V, M = _pack(sims)
    h = nb.nbody_create_batch(offs, [s[3] for s in sims])
    nb.nbody_set_state(h, X, V, M)
    best, ms = nb.nbody_autotune(h, 2)
    assert 0 <= best < nb.NBODY_NTUNE and nb.nbody_get_tuning(h) == best
    assert all(t > 0 for t in ms) and ms[best] == min(ms)
    xo = torch.empty_like(X)
    nb.nbody_get_state(h, xo, None)
    assert torch.equal(xo, X)   # tuning does not advance the state
    nb.nbody_destroy(h)


def test_fused_step_matches_separate_kernels():
    """Launch shape 0 (j-chunks of 4096: every member here takes one chunk)
    runs the fused pair + update step; shape 1 (chunks of 2048: the 2600
    member takes two) runs separate pair and update kernels.  Same
    arithmetic up to the order of the FP64 chunk sums."""
    sims = _members()
    fused = _run_batch(sims, 30, tuning=0)
    split = _run_batch(sims, 30, tuning=1)
    for xa, xb, s in zip(fused, split, sims):
        scale = 1.0 if s[4].ext == 0 else C1.a_prog
        assert np.abs(xa - xb).max() / scale <= 1e-10


def test_batch_tiny_and_ragged_members():
    """Members of 1, 2 and 1025 particles (one lone particle feels only the
    field; a 1025-member pads to 2048) in both the fused and the split step
    against the oracle."""
    pot = C1.pot
    sims = []
    for k, n in enumerate((1, 2, 1025)):
        x, v, m = plummer_sphere(max(n, 2), 60 + k, C1.G, C1.M_prog, C1.a_prog, center=C1.X0,
                                 velocity=C1.V0)
        x, v, m = x[:n], v[:n], m[:n]
        p = nb.make_params(C1.G, C1.eps, 0.5, ext_flags=3, nfw_M=pot.nfw_M, nfw_rs=pot.nfw_rs,
                           mn_M=pot.mn_M, mn_a=pot.mn_a, mn_b=pot.mn_b, center=C1.X0,
                           center_vel=C1.V0, center_mode=nb.NBODY_CENTER_GUIDE)
        ph = orc.Physics(G=C1.G, eps=C1.eps, ext=orc.NFW | orc.MN, nfw_M=pot.nfw_M,
                         nfw_rs=pot.nfw_rs, mn_M=pot.mn_M, mn_a=pot.mn_a, mn_b=pot.mn_b)
        sims.append((x, v, m, p, ph))
    for tuning in (0, 1, nb.NBODY_NTUNE - 1):
        got = _run_batch(sims, 20, tuning=tuning)
        for (x, v, m, p, ph), xb in zip(sims, got):
            xr, _ = orc.integrate(ph, x, v, m, p.dt, 20)
            assert_positions_close(xb, xr, ph)


@pytest.mark.parametrize("uneq", [False, True])
def test_batch_adjoint_matches_oracle(uneq):
    """The batched reverse sweep of a recorded run (three members of uneven
    size with their own dt, potential and centre) against the oracle's
    adjoint of each member: dL/dx0, dL/dv0 norm-wise and every parameter
    gradient at 1e-4; repeated sweeps give the same bits; host arrays too."""
    sims = _members()
    if uneq:   # unequal masses in one member: the general VJP kernel
        x, v, m, p, ph = sims[1]
        sims[1] = (x, v, m * np.linspace(0.5, 1.5, len(m)), p, ph)
    # and a tiny member (7 particles in a 1024-row pad)
    x, v, m = plummer_sphere(7, 33, 1.0, 1.0, 1.0)
    sims.append((x, v, m, nb.make_params(1.0, 0.05, 1e-3), orc.Physics(G=1.0, eps=0.05)))
    for s in sims:
        s[3].checkpoint_every = 1
    steps = 25
    offs, X, V, M = _pack(sims)
    h = nb.nbody_create_batch(offs, [s[3] for s in sims])
    try:
        nb.nbody_set_state(h, X, V, M)
        with pytest.raises(nb.NBodyError) as e:      # nothing recorded yet
            nb.nbody_vjp_batch(h, len(sims), X, V)
        assert e.value.code == nb.NBODY_ESTATE
        nb.nbody_integrate(h, steps)
        rng = np.random.default_rng(17)
        wx = rng.normal(size=(int(offs[-1]), 3))
        wv = rng.normal(size=(int(offs[-1]), 3))
        WX, WV = torch.tensor(wx.T.copy(), device=DEV), torch.tensor(wv.T.copy(), device=DEV)
        x0b, v0b = torch.empty_like(X), torch.empty_like(X)
        tb = nb.nbody_vjp_batch(h, len(sims), WX, WV, x0b, v0b)
        x0b2, v0b2 = torch.empty_like(X), torch.empty_like(X)
        tb2 = nb.nbody_vjp_batch(h, len(sims), WX, WV, x0b2, v0b2)
        assert torch.equal(x0b, x0b2) and torch.equal(v0b, v0b2) and np.array_equal(tb, tb2)
        hx = np.empty((3, int(offs[-1])))
        tb3 = nb.nbody_vjp_batch(h, len(sims), wx.T.copy(), wv.T.copy(), hx, None)
        assert np.array_equal(hx, x0b.cpu().numpy()) and np.array_equal(tb3, tb)
        # cotangents 2^100 larger (their FP32 copies would overflow in the pair
        # VJP unscaled): the per-simulation power-of-two scaling stages the
        # same FP32 values, so every result is exactly 2^100 larger
        big = 2.0 ** 100
        x0b4, v0b4 = torch.empty_like(X), torch.empty_like(X)
        tb4 = nb.nbody_vjp_batch(h, len(sims), WX * big, WV * big, x0b4, v0b4)
        assert torch.equal(x0b4, x0b * big) and torch.equal(v0b4, v0b * big)
        assert np.array_equal(tb4, tb * big)
        assert nb.nbody_get_status(h) == 0
    finally:
        nb.nbody_destroy(h)
    gx, gv = x0b.cpu().numpy().T, v0b.cpu().numpy().T
    for k, (x, v, m, p, ph) in enumerate(sims):
        sl = slice(int(offs[k]), int(offs[k + 1]))
        r = orc.vjp(ph, x, v, m, p.dt, steps, wx[sl], wv[sl])
        for got, ref in ((gx[sl], r["x0bar"]), (gv[sl], r["v0bar"])):
            assert per_particle_err(got, ref) <= 1e-4, k
        assert tb[k, 0] == pytest.approx(r["dt_bar"], rel=1e-4)
        assert tb[k, 1] == pytest.approx(np.dot(m, r["mbar"]), rel=1e-4)
        if ph.ext:
            ref = [r["nfw_M_bar"], r["mn_M_bar"], r["nfw_rs_bar"], r["mn_a_bar"], r["mn_b_bar"]]
            assert tb[k, 2:7] == pytest.approx(ref, rel=1e-4), k
        else:
            assert np.all(tb[k, 2:] == 0.0)
        assert tb[k, 7] == 0.0


def test_batch_adjoint_needs_consistent_tape_requests():
    sims = _members()
    sims[0][3].checkpoint_every = 1
    offs, X, V, M = _pack(sims)
    with pytest.raises(nb.NBodyError) as e:
        nb.nbody_create_batch(offs, [s[3] for s in sims])
    assert e.value.code == nb.NBODY_EINVAL


def test_batch_adjoint_single_member_single_step():
    """The smallest recorded run (one simulation, one step) and a run of no
    recorded steps after a plain one: against the oracle, and ESTATE when the
    last run did not record."""
    x, v, m = plummer_sphere(50, 34, 1.0, 1.0, 1.0)
    p = nb.make_params(1.0, 0.05, 1e-2, checkpoint_every=1)
    h = nb.nbody_create_batch([0, 50], [p])
    try:
        X = torch.tensor(x.T.copy(), device=DEV)
        V = torch.tensor(v.T.copy(), device=DEV)
        nb.nbody_set_state(h, X, V, torch.tensor(m, device=DEV))
        nb.nbody_integrate(h, 1)
        # the state into device and into host arrays: the same bits
        xd, xh = torch.empty_like(X), np.empty((3, 50))
        vh = np.empty((3, 50))
        nb.nbody_get_state(h, xd, None)
        nb.nbody_get_state(h, xh, vh)
        assert np.array_equal(xh, xd.cpu().numpy()) and np.all(np.isfinite(vh))
        rng = np.random.default_rng(5)
        wx, wv = rng.normal(size=(50, 3)), rng.normal(size=(50, 3))
        x0b, v0b = torch.empty_like(X), torch.empty_like(X)
        tb = nb.nbody_vjp_batch(h, 1, torch.tensor(wx.T.copy(), device=DEV),
                                torch.tensor(wv.T.copy(), device=DEV), x0b, v0b)
        r = orc.vjp(orc.Physics(G=1.0, eps=0.05), x, v, m, 1e-2, 1, wx, wv)
        for got, ref in ((x0b.cpu().numpy().T, r["x0bar"]), (v0b.cpu().numpy().T, r["v0bar"])):
            assert per_particle_err(got, ref) <= 1e-5
        assert tb[0, 0] == pytest.approx(r["dt_bar"], rel=1e-5)
        assert tb[0, 1] == pytest.approx(np.dot(m, r["mbar"]), rel=1e-5)
        # a new state invalidates the recorded run
        nb.nbody_set_state(h, X, V, torch.tensor(m, device=DEV))
        with pytest.raises(nb.NBodyError) as e:
            nb.nbody_vjp_batch(h, 1, None, None)
        assert e.value.code == nb.NBODY_ESTATE
    finally:
        nb.nbody_destroy(h)

"""MMD kernels vs the FP64 oracle, through the C ABI (needs a GB300).

Tolerances: the kernel values are summed in FP32 within 512-point tiles
(ex2.approx, relative error ~2^-22) and in FP64 across tiles; each of the
three terms of MMD^2 is at most n_sigma, so the loss is compared with an
absolute bound of 1e-5 * n_sigma and the gradient point by point at 1e-4
(relative to each point's gradient, floored at 1e-3 of the rms).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mmd as om  # noqa: E402
from paper_2511_22468_gb300 import nbody as nb  # noqa: E402
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


def stream_like(n, seed, shift=0.0):
    """A seeded elongated cloud in kpc and kpc/Myr (a stream-like shape:
    long along one axis, thin across, a velocity gradient along it)."""
    rng = np.random.default_rng(seed)
    t = rng.uniform(-1, 1, n)
    x = np.stack([8.0 * t + rng.normal(0, 0.2, n), 3.0 * t ** 2 + rng.normal(0, 0.1, n),
                  rng.normal(0, 0.15, n)], axis=1) + np.array([-5.0, 2.0, 9.0]) + shift
    v = np.stack([0.2 + 0.02 * t, -0.05 * t + rng.normal(0, 0.003, n),
                  rng.normal(0, 0.004, n)], axis=1) + 0.01 * shift
    return x, v


def soa(a):
    return torch.tensor(np.ascontiguousarray(np.asarray(a, np.float64).T), device=DEV)


@pytest.mark.parametrize("n,m,sig", [(600, 700, [1.0]), (1000, 1000, [0.5, 1.0, 2.0]),
                                     (2500, 1800, [0.3, 0.6, 1.2, 2.4]),
                                     (5, 3, [1.0, 2.0]), (513, 511, [0.7])])
def test_mmd_matches_oracle(n, m, sig):
    xs, vs = stream_like(n, 1, shift=0.3)
    xt, vt = stream_like(m, 2)
    X, Y = om.cloud(xs, vs), om.cloud(xt, vt)
    L_ref, g_ref = om.mmd2_grad(X, Y, sig)
    h = nb.nbody_mmd_create(n, 1, soa(xt), soa(vt), sig)
    try:
        xb = torch.empty((3, n), dtype=torch.float64, device=DEV)
        vb = torch.empty_like(xb)
        L = nb.nbody_mmd_eval(h, soa(xs), soa(vs), xb, vb)
        assert abs(L - L_ref) <= 1e-5 * len(sig)
        g = np.concatenate([xb.cpu().numpy().T, vb.cpu().numpy().T], axis=1)
        assert per_particle_err(g, g_ref) <= 1e-4
        mu, sc = nb.nbody_mmd_target_stats(h)
        mu_ref, sc_ref = om.target_stats(Y)
        np.testing.assert_allclose(mu, mu_ref, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(sc, sc_ref, rtol=1e-10)
        # bitwise reproducible, and host arrays give the same result
        L2 = nb.nbody_mmd_eval(h, np.ascontiguousarray(xs.T), np.ascontiguousarray(vs.T))
        assert L2 == L
    finally:
        nb.nbody_mmd_destroy(h)


def test_batched_sets_match_oracle():
    n, m, sets, sig = 1000, 1200, 7, [0.5, 1.0, 2.0]
    xt, vt = stream_like(m, 3)
    Y = om.cloud(xt, vt)
    clouds = [stream_like(n, 10 + b, shift=0.1 * b) for b in range(sets)]
    X = torch.cat([soa(c[0]) for c in clouds], dim=1).contiguous()
    V = torch.cat([soa(c[1]) for c in clouds], dim=1).contiguous()
    h = nb.nbody_mmd_create(n, 16, soa(xt), soa(vt), sig)
    try:
        out = torch.empty(sets, dtype=torch.float64, device=DEV)
        nb.nbody_mmd_eval_batch(h, sets, X, V, out)
        got = out.cpu().numpy()
        for b, (xs, vs) in enumerate(clouds):
            ref = om.mmd2(om.cloud(xs, vs), Y, sig)
            assert abs(got[b] - ref) <= 1e-5 * len(sig)
            single = nb.nbody_mmd_eval(h, soa(xs), soa(vs))
            assert got[b] == pytest.approx(single, rel=1e-12, abs=1e-15)
        with pytest.raises(nb.NBodyError) as e:
            nb.nbody_mmd_eval_batch(h, 17, X, V, out)
        assert e.value.code == nb.NBODY_EINVAL
    finally:
        nb.nbody_mmd_destroy(h)


def test_identical_cloud_and_single_points():
    xt, vt = stream_like(1500, 4)
    h = nb.nbody_mmd_create(1500, 1, soa(xt), soa(vt), [1.0, 2.0])
    try:
        assert abs(nb.nbody_mmd_eval(h, soa(xt), soa(vt))) < 1e-12
    finally:
        nb.nbody_mmd_destroy(h)
    # one point each, explicit scale: MMD^2 = 2 - 2/e for d^2 = 2, sigma = 1
    a = np.array([[1.0, 2.0, 3.0, 0.0, 0.0, 0.0]])
    b = a + np.array([[2.0, 1.0, 0.0, 0.0, 0.0, 0.0]])
    sc = [2.0, 1.0, 1.0, 3.0, 1.0, 1.0]
    h = nb.nbody_mmd_create(1, 1, soa(b[:, :3]), soa(b[:, 3:]), [1.0], scale=sc)
    try:
        L = nb.nbody_mmd_eval(h, soa(a[:, :3]), soa(a[:, 3:]))
        assert L == pytest.approx(1.2642411176571153, abs=2e-6)
    finally:
        nb.nbody_mmd_destroy(h)


def test_mmd_errors():
    xt, vt = stream_like(10, 5)
    for kw in (dict(sigmas=[]), dict(sigmas=[1.0, -1.0]), dict(sigmas=[1.0] * 5)):
        with pytest.raises(nb.NBodyError) as e:
            nb.nbody_mmd_create(10, 1, soa(xt), soa(vt), **kw)
        assert e.value.code == nb.NBODY_EINVAL
    # a target without spread needs an explicit scale
    one = soa(xt[:1])
    with pytest.raises(nb.NBodyError) as e:
        nb.nbody_mmd_create(10, 1, one, soa(vt[:1]), [1.0])
    assert e.value.code == nb.NBODY_EINVAL


@pytest.mark.parametrize("n,m2,sets,targets,sig", [(1000, 1000, 6, 5, [0.5, 1.0, 2.0]),
                                                   (700, 513, 3, 4, [1.0]),
                                                   (5, 9, 2, 3, [0.3, 0.6, 1.2, 2.4])])
def test_cross_targets_match_oracle(n, m2, sets, targets, sig):
    """Many clouds against many perturbed realisations of the observation,
    in the evaluator's units (its own target's standardisation): each loss
    against the oracle's MMD^2 with that standardisation."""
    from paper_2511_22468_gb300.inputs import perturbed_clouds
    xt, vt = stream_like(m2, 6)
    Y = om.cloud(xt, vt)
    mu, s = om.target_stats(Y)
    rx, rv = perturbed_clouds(xt, vt, 0.1, 2e-3, targets, seed=7)
    clouds = [stream_like(n, 20 + b, shift=0.05 * b) for b in range(sets)]
    X = torch.cat([soa(c[0]) for c in clouds], dim=1).contiguous()
    V = torch.cat([soa(c[1]) for c in clouds], dim=1).contiguous()
    TY = torch.cat([soa(rx[t]) for t in range(targets)], dim=1).contiguous()
    TV = torch.cat([soa(rv[t]) for t in range(targets)], dim=1).contiguous()
    h = nb.nbody_mmd_create(n, sets, soa(xt), soa(vt), sig)
    try:
        out = torch.empty(targets * sets, dtype=torch.float64, device=DEV)
        nb.nbody_mmd_eval_cross(h, sets, X, V, targets, m2, TY, TV, out)
        got = out.cpu().numpy().reshape(targets, sets)
        for t in range(targets):
            Yt = om.cloud(rx[t], rv[t])
            for b, (xs, vs) in enumerate(clouds):
                ref = om.mmd2(om.cloud(xs, vs), Yt, sig, mu, s)
                assert abs(got[t, b] - ref) <= 1e-5 * len(sig), (t, b)
        # against the evaluator's own target it is the batched evaluation
        # (same terms, another summation order)
        one = torch.empty(sets, dtype=torch.float64, device=DEV)
        nb.nbody_mmd_eval_cross(h, sets, X, V, 1, m2, soa(xt), soa(vt), one)
        ref1 = torch.empty(sets, dtype=torch.float64, device=DEV)
        nb.nbody_mmd_eval_batch(h, sets, X, V, ref1)
        assert torch.allclose(one, ref1, rtol=0, atol=1e-6 * len(sig))
        # host arrays give the same bits; repeated calls too
        host = np.empty(targets * sets)
        nb.nbody_mmd_eval_cross(h, sets, X.cpu().numpy(), V.cpu().numpy(), targets, m2,
                                TY.cpu().numpy(), TV.cpu().numpy(), host)
        assert np.array_equal(host, out.cpu().numpy())
        with pytest.raises(nb.NBodyError) as e:
            nb.nbody_mmd_eval_cross(h, 0, X, V, targets, m2, TY, TV, out)
        assert e.value.code == nb.NBODY_EINVAL
    finally:
        nb.nbody_mmd_destroy(h)


def test_cross_full_size_sampled():
    """The bootstrap's full size (10^4 clouds of 1000 points against 1000
    realisations of 1000 points, the launch configuration of the benchmark's
    bootstrap): sampled (cloud, realisation) losses against the oracle."""
    from paper_2511_22468_gb300.inputs import perturbed_clouds
    n = m = 1000
    sets, targets, sig = 10000, 1000, [0.5, 1.0, 2.0]
    xb, vb = stream_like(n, 41)
    rng = np.random.default_rng(42)
    f = 1.0 + 0.05 * rng.normal(size=(sets, 1, 1))
    dx = 0.3 * rng.normal(size=(sets, 1, 3))
    cx = xb[None] * f + dx                        # (sets, n, 3)
    cv = vb[None] * f + 0.01 * dx
    rx, rv = perturbed_clouds(xb, vb, 0.05 * xb.std(axis=0), 0.05 * vb.std(axis=0), targets,
                              seed=43)
    Y = om.cloud(xb, vb)
    mu, s = om.target_stats(Y)
    to_dev = lambda a: torch.tensor(  # noqa: E731
        np.ascontiguousarray(a.transpose(2, 0, 1).reshape(3, -1)), device=DEV)
    h = nb.nbody_mmd_create(n, 1, soa(xb), soa(vb), sig)
    try:
        out = torch.empty(targets * sets, dtype=torch.float64, device=DEV)
        nb.nbody_mmd_eval_cross(h, sets, to_dev(cx), to_dev(cv), targets, m, to_dev(rx),
                                to_dev(rv), out)
        got = out.cpu().numpy().reshape(targets, sets)
    finally:
        nb.nbody_mmd_destroy(h)
    assert np.all(np.isfinite(got))
    for t, b in [(0, 0), (999, 9999), (17, 5003), (500, 1), (3, 7777), (998, 2)]:
        ref = om.mmd2(om.cloud(cx[b], cv[b]), om.cloud(rx[t], rv[t]), sig, mu, s)
        assert abs(got[t, b] - ref) <= 1e-5 * len(sig), (t, b, got[t, b], ref)

"""The mock-stream pipeline on the GPU (backward orbit, Plummer shift,
n-body run, sky projection, soft histogram, loss) and its adjoint against
the FP64 oracle (needs a GB300).

Tolerances: density element-wise 1e-8 absolute (densities are O(1e-3));
loss 1e-4 relative; each dL/dTheta component 1e-4 relative of the oracle
adjoint and of the oracle's central differences (Richardson).  dL/dt_end is
the difference of two parts, through the forward run's dt and through the
backward orbit's -dt, which cancel to first order (the centre of mass comes
back to X0); its error is bounded by 1e-4 of the sum of the parts' sizes.
"""

import dataclasses
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import stream as ostream  # noqa: E402
from paper_2511_22468_gb300.configs import C1  # noqa: E402
from paper_2511_22468_gb300.inputs import plummer_unit  # noqa: E402

pytestmark = pytest.mark.gpu


def assert_grad_close(g, g_ref, parts):
    """1e-4 relative per component; dL/dt_end (the difference of the forward
    run's and the backward orbit's parts) to 1e-4 of the parts' sizes."""
    scale = np.abs(np.asarray(g_ref, float))
    scale[0] = abs(parts[0]) + abs(parts[1])
    err = np.abs(np.asarray(g) - g_ref) / scale
    assert np.all(err <= 1e-4), (g, g_ref, parts, err)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22468_gb300 import build, nbody
    build.build()
    nbody.lib()


def _case(n=384, t_acc=30.0, n_steps=60):
    cfg = dataclasses.replace(C1, n=n, t_acc=t_acc, n_steps=n_steps)
    xh, vh = plummer_unit(n, 1)
    return cfg, xh, vh


@pytest.mark.parametrize("K", [8, 60])
def test_stream_loss_and_gradient_match_oracle(K):
    from paper_2511_22468_gb300.stream import StreamModel
    cfg, xh, vh = _case()
    orc = ostream.StreamModel(cfg, xh, vh)
    truth = np.array(cfg.theta_true, float)
    target = orc.density(truth)
    th = truth * np.array([1.05, 0.9, 1.1, 0.95])
    L_ref, g_ref = orc.loss_and_grad(th, target)

    gpu = StreamModel(cfg, xh, vh, checkpoint_every=K)
    gpu.set_target(target)
    rho = gpu.density(th).cpu().numpy()
    np.testing.assert_allclose(rho, orc.density(th), rtol=0, atol=1e-8)
    L, g = gpu.loss_and_grad(th)
    assert L == pytest.approx(L_ref, rel=1e-4)
    assert_grad_close(g, g_ref, orc.t_end_parts)

    # against the oracle's central differences (Richardson-extrapolated)
    for k in range(4):
        h = 1e-4 * th[k]
        def f(s):
            t = th.copy()
            t[k] += s
            return orc.loss(t, target)
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        fd = (4 * d2 - d1) / 3
        tol = 1e-4 * (abs(fd) if k else sum(abs(p) for p in orc.t_end_parts))
        assert abs(g[k] - fd) <= tol, (k, g[k], fd)
    gpu.close()


def test_stream_autograd_function():
    from paper_2511_22468_gb300.stream import StreamLoss, StreamModel
    cfg, xh, vh = _case(n=256, t_acc=20.0, n_steps=40)
    orc = ostream.StreamModel(cfg, xh, vh)
    truth = np.array(cfg.theta_true, float)
    gpu = StreamModel(cfg, xh, vh, checkpoint_every=7)
    gpu.set_target(orc.density(truth))
    theta = torch.tensor(truth * np.array([0.95, 1.1, 0.9, 1.05]), dtype=torch.float64,
                         requires_grad=True)
    L = StreamLoss.apply(theta, gpu)
    L.backward()
    L_ref, g_ref = orc.loss_and_grad(theta.detach().numpy(), orc.density(truth))
    assert L.item() == pytest.approx(L_ref, rel=1e-4)
    assert_grad_close(theta.grad.numpy(), g_ref, orc.t_end_parts)
    # at the truth the loss and its gradient vanish up to the FP32 pair
    # sums' rounding (the target is the oracle's density)
    assert gpu.loss(truth) <= 1e-6 * L_ref
    assert np.all(np.abs(gpu.grad()) <= 1e-3 * np.abs(g_ref))
    gpu.close()


def test_stream_mmd_loss_and_gradient_match_oracle():
    """The point-cloud form (MMD^2 of the final phase-space cloud against a
    target cloud) through the pipeline's adjoint, against the oracle."""
    from oracle import mmd
    from paper_2511_22468_gb300.stream import StreamModel
    cfg, xh, vh = _case()
    orc = ostream.StreamModel(cfg, xh, vh)
    truth = np.array(cfg.theta_true, float)
    xt, vt = orc.final_state(truth)
    Y = mmd.cloud(xt, vt)
    sig = [0.5, 1.0, 2.0]
    th = truth * np.array([1.05, 0.9, 1.1, 0.95])
    L_ref, g_ref = orc.mmd_loss_and_grad(th, Y, sig)
    gpu = StreamModel(cfg, xh, vh, checkpoint_every=8)
    gpu.set_target_cloud(xt.T.copy(), vt.T.copy(), sig)
    L, g = gpu.loss_and_grad(th)
    assert abs(L - L_ref) <= 1e-5 * len(sig) and L == pytest.approx(L_ref, rel=1e-3)
    assert_grad_close(g, g_ref, orc.t_end_parts)
    # the GPU's own final state at the truth reproduces the target cloud
    xg, vg = gpu.final_state(list(truth))
    assert np.max(np.abs(xg.cpu().numpy().T - xt)) <= 1e-6 * np.max(np.abs(xt))
    assert gpu.loss(list(truth)) < 1e-9
    # a new target of the same size is taken in place: the same bits as a
    # fresh pipeline given that target
    xt2, vt2 = orc.final_state(truth * 1.02)
    gpu.set_target_cloud(xt2.T.copy(), vt2.T.copy(), sig)
    L2, g2 = gpu.loss_and_grad(th)
    fresh = StreamModel(cfg, xh, vh, checkpoint_every=8)
    fresh.set_target_cloud(xt2.T.copy(), vt2.T.copy(), sig)
    L2f, g2f = fresh.loss_and_grad(th)
    fresh.close()
    assert L2 == L2f and np.array_equal(g2, g2f)
    # switching back to the density loss
    gpu.set_target(orc.density(truth))
    assert gpu.loss(list(th)) == pytest.approx(orc.loss(th, orc.density(truth)), rel=1e-4)
    gpu.close()


def test_stream_autotune_keeps_parity():
    """Tuned launch shapes of the pipeline's n-body kernels give the same
    loss and gradient as the oracle."""
    from paper_2511_22468_gb300.stream import StreamModel
    cfg, xh, vh = _case()
    orc = ostream.StreamModel(cfg, xh, vh)
    truth = np.array(cfg.theta_true, float)
    target = orc.density(truth)
    th = truth * np.array([1.05, 0.9, 1.1, 0.95])
    L_ref, g_ref = orc.loss_and_grad(th, target)
    gpu = StreamModel(cfg, xh, vh, checkpoint_every=8)
    gpu.set_target(target)
    gpu.autotune(list(th))
    L, g = gpu.loss_and_grad(th)
    assert L == pytest.approx(L_ref, rel=1e-4)
    assert_grad_close(g, g_ref, orc.t_end_parts)
    gpu.close()


def test_stream_batch_losses_and_gradients_match_oracle():
    """The pipeline for several parameter vectors at once, each member
    against its own target cloud in common units: every member's MMD^2 and
    dL/dtheta against the oracle's pipeline for that member."""
    from oracle import mmd
    from paper_2511_22468_gb300.stream import StreamBatch
    from paper_2511_22468_gb300.surrogate import descend_batch
    cfg, xh, vh = _case()
    orc = ostream.StreamModel(cfg, xh, vh)
    truth = np.array(cfg.theta_true, float)
    f_target = np.array([[1.0, 1.0, 1.0, 1.0], [1.1, 0.9, 1.0, 1.05], [0.95, 1.1, 1.05, 0.9]])
    f_theta = np.array([[1.05, 0.9, 1.1, 0.95], [1.0, 1.0, 0.95, 1.1], [0.9, 1.05, 1.0, 1.0]])
    targets = [orc.final_state(truth * f) for f in f_target]
    tx = np.stack([t[0] for t in targets])
    tv = np.stack([t[1] for t in targets])
    Y0 = mmd.cloud(tx[0], tv[0])
    mu, sc = mmd.target_stats(Y0)
    sig = [0.5, 1.0, 2.0]
    thetas = truth[None, :] * f_theta
    gpu = StreamBatch(cfg, xh, vh, tx, tv, sig, scale=sc)
    L, g = gpu.loss_and_grad(thetas)
    parts = gpu.grad_parts()
    for b in range(3):
        Yb = mmd.cloud(tx[b], tv[b])
        L_ref, g_ref = orc.mmd_loss_and_grad(thetas[b], Yb, sig, mu, sc)
        assert abs(L[b] - L_ref) <= 1e-5 * len(sig) and L[b] == pytest.approx(L_ref, rel=1e-3)
        # each component is the sum of two parts (n-body run and backward
        # orbit; velocity scaling and masses); dL/dt_end is held to 1e-4 of
        # its parts (reading of the t_end bound), dL/dM_Plummer to 1e-4.
        # dL/dM_NFW and dL/dM_MN: their parts cancel 50-540x here and both
        # depend on the common mode of the FP32 point-cloud cotangent (a sum
        # over the cloud that cancels to a few per cent), which shifts the
        # two parts in opposite directions; the bound adds 2e-5 of the
        # parts' sizes to 1e-4 of the component.  The component is the sum
        # of the reported parts, bit for bit.
        p1, p2 = orc.grad_parts
        gp = parts[b]
        np.testing.assert_array_equal(gp[0] + gp[1], g[b])
        scale = 1e-4 * np.abs(g_ref)
        scale[0] = 1e-4 * (abs(p1[0]) + abs(p2[0]))
        scale[2:] += 2e-5 * (np.abs(p1[2:]) + np.abs(p2[2:]))
        assert np.all(np.abs(g[b] - g_ref) <= scale), (b, g[b], g_ref, p1, p2)
    # the same call again gives the same bits; the loss alone agrees
    L2, g2 = gpu.loss_and_grad(thetas)
    assert np.array_equal(L, L2) and np.array_equal(g, g2)
    assert np.array_equal(gpu.loss(thetas), L)
    # a member at its own target's parameters has zero loss (to the loss
    # tolerance: the target is the oracle's cloud, the kernel sums are FP32)
    L0, _ = gpu.loss_and_grad(truth[None, :] * f_target)
    assert np.all(np.abs(L0) <= 1e-5 * len(sig)) and np.all(np.abs(L0) < 1e-3 * L)
    # batched descent: the best loss of every member never increases
    best, Lb, trace = descend_batch(gpu, thetas, truth, 0.3, iters=3)
    assert trace.shape == (4, 3) and np.all(np.diff(trace, axis=0) <= 0.0)
    assert np.all(Lb <= L) and np.array_equal(Lb, trace[-1])
    gpu.close()


def test_stream_batch_isolates_a_failing_member():
    """A member whose run leaves the finite range (a halo mass of 1e300)
    gets loss +inf and a NaN gradient; the other members get the bits they
    get without it, and the next call is clean again."""
    from paper_2511_22468_gb300.stream import StreamBatch
    cfg, xh, vh = _case()
    orc = ostream.StreamModel(cfg, xh, vh)
    truth = np.array(cfg.theta_true, float)
    xt, vt = orc.final_state(truth)
    tx, tv = np.stack([xt] * 3), np.stack([vt] * 3)
    thetas = truth[None, :] * np.array([[1.05, 0.9, 1.1, 0.95], [1.0, 1.0, 1.0, 1.0],
                                        [0.95, 1.05, 1.0, 1.02]])
    gpu = StreamBatch(cfg, xh, vh, tx, tv)
    L, g = gpu.loss_and_grad(thetas)
    assert np.all(np.isfinite(L)) and np.all(np.isfinite(g))
    bad = thetas.copy()
    bad[1, 2] = 1e300
    Lb, gb = gpu.loss_and_grad(bad)
    assert Lb[1] == np.inf and np.all(np.isnan(gb[1]))
    assert Lb[0] == L[0] and Lb[2] == L[2]
    assert np.array_equal(gb[[0, 2]], g[[0, 2]])
    L2, g2 = gpu.loss_and_grad(thetas)
    assert np.array_equal(L2, L) and np.array_equal(g2, g)
    gpu.close()


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("steps", [200])
def test_stream_pipeline_at_workload_size(steps):
    """The GD-1-like stream workload at its own size, N = 10^4, over `steps`
    steps of 0.5 Myr, in the launch shapes the pipeline's autotuner picks at
    that size, against the oracle's values stored by
    tests/golden/make_stream_n1e4.py (the oracle alone computes them):
    density per bin 1e-8 absolute, loss 1e-4 relative, dL/dTheta per
    component 1e-4 relative of the oracle adjoint (dL/dt_end: of its parts)
    and of the oracle's Richardson central differences."""
    from paper_2511_22468_gb300 import nbody as nb
    from paper_2511_22468_gb300.stream import StreamModel
    g = json.load(open(os.path.join(GOLDEN, "stream_n1e4_s%d.json" % steps)))
    cfg = dataclasses.replace(C1, t_acc=g["t_end_true"], n_steps=g["n_steps"])
    assert cfg.n == g["n"] and cfg.seed == g["seed"]
    xh, vh = plummer_unit(cfg.n, cfg.seed)
    fp = g["inputs"]
    np.testing.assert_allclose([np.abs(xh).sum(), np.abs(vh).sum()],
                               [fp["sum_abs_x"], fp["sum_abs_v"]], rtol=1e-12)
    np.testing.assert_allclose(xh[fp["rows"]], fp["x_rows"], rtol=1e-12)
    np.testing.assert_allclose(vh[fp["rows"]], fp["v_rows"], rtol=1e-12)
    th = np.array(g["theta"])
    gpu = StreamModel(cfg, xh, vh)
    gpu.set_target(np.array(g["target_density"]).reshape(cfg.nb1, cfg.nb2))
    gpu.autotune(list(th))
    shapes = [nb.nbody_stream_get_pair_shape(gpu.h, k) for k in (0, 1)]
    rho = gpu.density(th).cpu().numpy().ravel()
    np.testing.assert_allclose(rho, g["density"], rtol=0, atol=1e-8, err_msg=str(shapes))
    L, grad = gpu.loss_and_grad(th)
    assert L == pytest.approx(g["loss"], rel=1e-4), shapes
    assert_grad_close(grad, np.array(g["grad"]), g["t_end_parts"])
    fd = np.array(g["grad_fd_richardson"])
    scale = np.abs(fd)
    scale[0] = sum(abs(p) for p in g["t_end_parts"])
    assert np.all(np.abs(grad - fd) <= 1e-4 * scale), (grad, fd, shapes)
    gpu.close()

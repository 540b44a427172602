"""Grid-search stage with the point-cloud loss against the oracle (needs a
GB300): batched initial states, batched simulation of every grid point and
the batched MMD^2 ranking.

Tolerances: initial states 1e-12 relative (FP64 on both sides); grid
losses 1e-5 * n_sigma absolute plus 1e-3 relative (the FP32 pair sums of
the batched n-body run move the final clouds by ~1e-7 of their size)."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mmd as om  # noqa: E402
from oracle import stream as ostream  # noqa: E402
from paper_2511_22468_gb300 import nbody as nb  # noqa: E402
from paper_2511_22468_gb300.configs import C1  # noqa: E402
from paper_2511_22468_gb300.inputs import plummer_unit  # noqa: E402

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22468_gb300 import build
    build.build()
    nb.lib()


def _cfg(n=200, t_end=20.0, steps=40):
    return dataclasses.replace(C1, n=n, t_acc=t_end, n_steps=steps)


def test_batched_initial_states_match_oracle():
    from paper_2511_22468_gb300.stream import StreamModel
    cfg = _cfg()
    xh, vh = plummer_unit(cfg.n, 3)
    orc = ostream.StreamModel(cfg, xh, vh)
    gpu = StreamModel(cfg, xh, vh)
    rng = np.random.default_rng(0)
    thetas = np.array(cfg.theta_true)[None, :] * rng.uniform(0.7, 1.3, (5, 4))
    n, B = cfg.n, len(thetas)
    X = torch.empty((3, B * n), dtype=torch.float64, device=DEV)
    V, M = torch.empty_like(X), torch.empty(B * n, dtype=torch.float64, device=DEV)
    com = np.zeros((B, 6))
    nb.nbody_stream_initial_states(gpu.h, thetas, X, V, M, com)
    for b, th in enumerate(thetas):
        x0, v0, m = orc.initial_state(th)
        np.testing.assert_allclose(X[:, b * n:(b + 1) * n].cpu().numpy().T, x0, rtol=1e-12)
        np.testing.assert_allclose(V[:, b * n:(b + 1) * n].cpu().numpy().T, v0, rtol=1e-12,
                                   atol=1e-15)
        np.testing.assert_allclose(M[b * n:(b + 1) * n].cpu().numpy(), m, rtol=1e-15)
    gpu.close()


def test_grid_losses_match_oracle_and_rank_the_truth_first():
    from paper_2511_22468_gb300.gridsearch import GridSearch, regular_grid
    cfg = _cfg()
    xh, vh = plummer_unit(cfg.n, 4)
    orc = ostream.StreamModel(cfg, xh, vh)
    centre = np.array(cfg.theta_true, float)
    grid = regular_grid(centre, 0.3, 2)                     # 16 points
    theta_obs = grid[5]                                     # the truth is a grid point
    xt, vt = orc.final_state(theta_obs)
    Y = om.cloud(xt, vt)
    sig = [0.5, 1.0, 2.0]
    gs = GridSearch(cfg, xh, vh, xt.T.copy(), vt.T.copy(), sigmas=sig, batch=6)
    L = gs.losses(grid)                                     # 3 batches, the last ragged
    gs.close()
    ref = np.array([orc.mmd_loss(th, Y, sig) for th in grid])
    assert np.all(np.abs(L - ref) <= 1e-5 * len(sig) + 1e-3 * np.abs(ref)), (L, ref)
    assert int(np.argmin(L)) == 5 and L[5] < 1e-6


def test_bootstrap_cross_losses_match_oracle():
    """The kept grid clouds scored against perturbed realisations of the
    observation (in the observation's standardisation) equal the oracle's
    MMD^2 of the oracle's clouds; the noise-free realisation reproduces the
    grid losses."""
    from paper_2511_22468_gb300.gridsearch import GridSearch, regular_grid
    from paper_2511_22468_gb300.inputs import perturbed_clouds
    cfg = _cfg()
    xh, vh = plummer_unit(cfg.n, 4)
    orc = ostream.StreamModel(cfg, xh, vh)
    centre = np.array(cfg.theta_true, float)
    grid = regular_grid(centre, 0.3, 2)
    xt, vt = orc.final_state(grid[5])
    Y = om.cloud(xt, vt)
    mu, s = om.target_stats(Y)
    sig = [0.5, 1.0, 2.0]
    rx, rv = perturbed_clouds(xt, vt, 0.05, 1e-3, 3, seed=11)
    rx = np.concatenate([xt[None], rx])                    # realisation 0: no noise
    rv = np.concatenate([vt[None], rv])
    gs = GridSearch(cfg, xh, vh, xt.T.copy(), vt.T.copy(), sigmas=sig, batch=6,
                    keep_clouds=len(grid))
    L = gs.losses(grid)
    LB = gs.cross_losses(len(grid), rx, rv)
    gs.close()
    assert LB.shape == (4, len(grid))
    assert np.all(np.abs(LB[0] - L) <= 1e-6 * len(sig)), (LB[0], L)
    clouds = [om.cloud(*orc.final_state(th)) for th in grid]
    for r in range(4):
        Yr = om.cloud(rx[r], rv[r])
        ref = np.array([om.mmd2(c, Yr, sig, mu, s) for c in clouds])
        assert np.all(np.abs(LB[r] - ref) <= 1e-5 * len(sig) + 1e-3 * np.abs(ref)), (r, LB[r], ref)


"""What the trained surrogate and the batched grid stage gain over the
prior centre (needs a GB300), on the recovery workload (N = 1e4, 100 Myr,
the point-cloud loss) with a reduced training set (768 simulations from the
batched kernel).  The surrogate's inverted start has at most half the prior
centre's error in t_end, M_Plummer and M_NFW (the binned density at this
horizon carries almost no information on the disk mass M_MN) and a lower
simulator loss; the batched grid stage's start has at most half the prior
centre's error max_k |theta_k / theta_obs_k - 1| over all four parameters
and a lower loss."""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22468_gb300 import build, nbody
    build.build()
    nbody.lib()


def test_warm_starts_reduce_parameter_error():
    from paper_2511_22468_gb300.configs import C1, C4
    from paper_2511_22468_gb300.inputs import plummer_unit, uniform_factors
    from paper_2511_22468_gb300.stream import StreamBatch, StreamModel
    from paper_2511_22468_gb300.surrogate import (DENSITY_SCALE, EnsembleDensities, Surrogate,
                                                  from_u)
    from paper_2511_22468_gb300.warmstart import F_OBS, SIGMAS, pattern_search
    n, t_end = 10000, 100.0
    cfg = dataclasses.replace(C1, n=n, t_acc=t_end, n_steps=200, phi1_deg=(-1.0, 1.0),
                              phi2_deg=(-0.5, 0.5))
    xh, vh = plummer_unit(n, cfg.seed)
    centre = np.array(cfg.theta_true)
    obs = centre * np.array(F_OBS)

    def err(th, k=4):
        return float(np.max(np.abs(np.asarray(th)[:k] / obs[:k] - 1.0)))

    model = StreamModel(cfg, xh, vh)
    xt, vt = model.final_state(list(obs))
    rho = model.density(list(obs)).cpu().numpy().ravel()
    model.set_target_cloud(xt, vt, SIGMAS)
    L_centre = model.loss(list(centre))

    gen = EnsembleDensities(cfg, xh, vh)
    f = uniform_factors(896, C4.width, 4, 12345)
    Y = gen.densities(centre * f) * DENSITY_SCALE
    gen.close()
    U = (f - 1.0) / C4.width
    net = Surrogate(seed=1)
    hist = net.fit(U[:768], Y[:768], epochs=600, lr=1e-3, U_val=U[768:], Y_val=Y[768:],
                   log_every=100)
    assert hist[-1]["val_mse"] < 0.5 * hist[0]["val_mse"]
    u0, _ = net.invert(rho * DENSITY_SCALE)
    theta0 = from_u(u0, centre, C4.width)
    net.close()
    assert err(theta0, 3) < 0.5 * err(centre, 3)
    assert model.loss(list(theta0)) < L_centre

    X, V = xt.cpu().numpy().T, vt.cpu().numpy().T
    sb = StreamBatch(cfg, xh, vh, np.stack([X] * 81), np.stack([V] * 81), SIGMAS)
    grid = pattern_search(sb, centre, C4.width, obs, 0.0, s0=0.37, max_calls=4)
    sb.close()
    assert err(grid[-1]["theta"]) < 0.5 * err(centre)
    assert model.loss(grid[-1]["theta"]) < L_centre
    model.close()

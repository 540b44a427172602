"""What the trained surrogate gains over the method without it (needs a
GB300): on a reduced stream workload (N = 2000, 200 Myr, 768 training
simulations from the batched kernel), the network's inverted start has a
lower simulator loss than the prior centre, and gradient descent from it
reaches a lower loss within the same number of simulator gradients."""
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


def test_surrogate_warm_start_beats_prior_centre():
    from paper_2511_22468_gb300.configs import C1, C4
    from paper_2511_22468_gb300.inputs import plummer_unit, uniform_factors
    from paper_2511_22468_gb300.stream import StreamModel
    from paper_2511_22468_gb300.surrogate import (DENSITY_SCALE, EnsembleDensities, Surrogate,
                                                  descend, from_u)
    from paper_2511_22468_gb300.warmstart import F_OBS
    n, t_end = 2000, 200.0
    cfg = dataclasses.replace(C1, n=n, t_acc=t_end, n_steps=400)
    xh, vh = plummer_unit(n, cfg.seed)
    centre = np.array(cfg.theta_true)
    obs = centre * np.array(F_OBS)
    model = StreamModel(cfg, xh, vh)
    target = model.density(obs)
    model.set_target(target)
    gen = EnsembleDensities(cfg, xh, vh)
    f = uniform_factors(896, C4.width, 4, 12345)
    Y = gen.densities(centre * f) * DENSITY_SCALE
    gen.close()
    U = (f - 1.0) / C4.width
    net = Surrogate(seed=1)
    hist = net.fit(U[:768], Y[:768], epochs=600, lr=1e-3, U_val=U[768:], Y_val=Y[768:],
                   log_every=100)
    assert hist[-1]["val_mse"] < 0.5 * hist[0]["val_mse"]
    u0, _ = net.invert(target.cpu().numpy() * DENSITY_SCALE)
    theta0 = from_u(u0, centre, C4.width)
    net.close()
    L_centre = model.loss(centre)
    L_warm = model.loss(theta0)
    assert L_warm < 0.5 * L_centre
    plain = descend(model, centre, centre, C4.width, max_iters=8)
    warm = descend(model, theta0, centre, C4.width, max_iters=8)
    assert warm[-1]["loss"] < plain[-1]["loss"]
    model.close()

"""Orbit fitting and the Fisher matrix (Sec. 2.2.2) against the oracle (needs
a GB300).  Observations come from the oracle's orbit at the true
parameters.  Tolerances: arc points and chi^2 1e-10 relative (FP64 on both
sides, different operation order); the dual-number gradient and
Gauss-Newton matrix 1e-5 of the oracle's central differences; the Fisher
matrix 2e-3 of the oracle's
second differences; the exact Hessian (second-order duals) equals the
Gauss-Newton matrix to 1e-9 where the residuals vanish."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import orbitfit as of  # noqa: E402
from paper_2511_22468_gb300 import nbody as nb  # noqa: E402
from paper_2511_22468_gb300.configs import C1, G_KPC_MSUN_MYR  # noqa: E402

pytestmark = pytest.mark.gpu

VSUN = np.array([12.9, 245.6, 7.78]) * of.KMS
TRUTH = np.array([1e12, 16.0, 6.8e10, 3.0, 0.28])
SIG = np.array([math.radians(0.1), 0.05, 0.05, 1.0])
WIN = (math.radians(-60), math.radians(60))


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22468_gb300 import build
    build.build()
    nb.lib()


def _cfg():
    c = nb.nbody_orbitfit_cfg()
    c.G = G_KPC_MSUN_MYR
    c.X0[:] = list(C1.X0)
    c.V0[:] = list(C1.V0)
    c.observer[:] = list(C1.observer)
    c.observer_vel[:] = list(VSUN)
    c.phi1_lo, c.phi1_hi = WIN
    c.dt, c.t_max = 0.5, 2000.0
    c.sigma[:] = list(SIG)
    return c


def _oracle():
    return of.OrbitFit(G_KPC_MSUN_MYR, C1.X0, C1.V0, C1.observer, VSUN, WIN, 0.5, 2000.0)


def test_arc_chi2_gradient_and_gauss_newton():
    fit = _oracle()
    obs = of.mock_observations(fit, TRUTH, 40, (math.radians(-40), math.radians(40)), SIG, 1)
    h = nb.nbody_orbitfit_create(_cfg(), obs)
    try:
        th = TRUTH * np.array([1.1, 0.9, 1.05, 0.95, 1.2])
        arc = nb.nbody_orbitfit_arc(h, th)
        ref = fit.arc(th)
        assert arc.shape == ref.shape
        np.testing.assert_allclose(arc, ref, rtol=1e-10, atol=1e-12)
        chi2, g, A = nb.nbody_orbitfit_eval(h, [th, TRUTH])
        assert chi2[0] == pytest.approx(fit.chi2(th, obs, SIG), rel=1e-10)
        assert chi2[1] == pytest.approx(fit.chi2(TRUTH, obs, SIG), rel=1e-10)
        xi = np.log(th)
        gref = of.fd_gradient(lambda z: fit.chi2(np.exp(z), obs, SIG), xi, h=1e-5)
        np.testing.assert_allclose(g[0], gref, rtol=1e-5, atol=1e-6 * np.abs(gref).max())
        r = lambda z: fit.residuals(np.exp(z), obs, SIG)    # noqa: E731
        J = np.stack([(r(xi + e) - r(xi - e)) / 2e-6 for e in np.eye(5) * 1e-6], axis=1)
        np.testing.assert_allclose(A[0], J.T @ J, rtol=1e-5, atol=1e-6 * np.abs(J.T @ J).max())
    finally:
        nb.nbody_orbitfit_destroy(h)


def test_fisher_matrix_at_the_truth():
    """Noise-free observations: F = (1/2) d^2 chi^2 equals the Gauss-Newton
    matrix at the truth (zero residuals); both against the oracle."""
    fit = _oracle()
    obs = of.mock_observations(fit, TRUTH, 40, (math.radians(-40), math.radians(40)),
                               np.zeros(4), 0)
    h = nb.nbody_orbitfit_create(_cfg(), obs)
    try:
        F, Fg = nb.nbody_orbitfit_fisher(h, TRUTH)
        np.testing.assert_allclose(F, F.T, rtol=0, atol=1e-13 * np.abs(F).max())
        # zero residuals: the second-order terms vanish exactly
        np.testing.assert_allclose(F, Fg, rtol=1e-9, atol=1e-12 * np.abs(Fg).max())
        Href = of.fd_hessian(lambda z: fit.chi2(np.exp(z), obs, SIG), np.log(TRUTH), h=1e-3)
        np.testing.assert_allclose(F, 0.5 * Href, rtol=2e-3, atol=1e-5 * np.abs(F).max())
    finally:
        nb.nbody_orbitfit_destroy(h)
    # away from the truth, with noise: the residual curvature terms count
    obs = of.mock_observations(fit, TRUTH, 40, (math.radians(-40), math.radians(40)), SIG, 5)
    h = nb.nbody_orbitfit_create(_cfg(), obs)
    try:
        # a step small enough that no observation crosses an arc node (the
        # linear interpolation makes the Hessian piecewise continuous)
        th = TRUTH * np.array([1.2, 0.8, 0.9, 1.1, 1.5])
        F, Fg = nb.nbody_orbitfit_fisher(h, th)
        Href = of.fd_hessian(lambda z: fit.chi2(np.exp(z), obs, SIG), np.log(th), h=1e-5)
        # second differences at this step carry rounding noise of about
        # 4 eps chi^2 / h^2 in absolute terms
        noise = 4 * 2.2e-16 * fit.chi2(th, obs, SIG) / 1e-10
        np.testing.assert_allclose(F, 0.5 * Href, rtol=1e-4, atol=20 * noise)
        assert np.abs(F - Fg).max() > 1e-6 * np.abs(F).max()
    finally:
        nb.nbody_orbitfit_destroy(h)


def test_levenberg_marquardt_recovers_the_truth():
    """64 starts in [0.5, 2] theta_true on noise-free observations: the best
    start reaches chi^2 ~ 0 at the truth; on noisy observations the best
    start's chi^2 matches the oracle's there and is below the truth's."""
    fit = _oracle()
    rng = np.random.default_rng(4)
    starts = TRUTH[None, :] * np.exp(rng.uniform(np.log(0.5), np.log(2.0), (64, 5)))
    obs = of.mock_observations(fit, TRUTH, 40, (math.radians(-40), math.radians(40)),
                               np.zeros(4), 0)
    h = nb.nbody_orbitfit_create(_cfg(), obs)
    try:
        th, chi2, its = nb.nbody_orbitfit_lm(h, starts, max_iter=200, lo=TRUTH / 10, hi=TRUTH * 10)
        k = int(np.argmin(chi2))
        assert chi2[k] < 1e-8
        # distance from the truth in the metric of the Gauss-Newton matrix
        # (nearly free directions such as b_MN may stay off by more)
        _, _, A = nb.nbody_orbitfit_eval(h, [TRUTH])
        dxi = np.log(th[k] / TRUTH)
        assert dxi @ A[0] @ dxi < 1e-8
        np.testing.assert_allclose(th[k][[2, 3]], TRUTH[[2, 3]], rtol=1e-4)
        assert np.all(its <= 200)
    finally:
        nb.nbody_orbitfit_destroy(h)
    obs = of.mock_observations(fit, TRUTH, 40, (math.radians(-40), math.radians(40)), SIG, 2)
    h = nb.nbody_orbitfit_create(_cfg(), obs)
    try:
        th, chi2, its = nb.nbody_orbitfit_lm(h, starts, max_iter=200, lo=TRUTH / 10, hi=TRUTH * 10)
        k = int(np.argmin(chi2))
        assert chi2[k] == pytest.approx(fit.chi2(th[k], obs, SIG), rel=1e-10)
        # the estimate fits the noisy track at least as well as the truth, and
        # no start ends above where it began
        assert chi2[k] <= fit.chi2(TRUTH, obs, SIG)
        c0, _, _ = nb.nbody_orbitfit_eval(h, starts, want_grad=False, want_gn=False)
        assert np.all(chi2 <= c0)
    finally:
        nb.nbody_orbitfit_destroy(h)


def test_orbitfit_errors():
    fit = _oracle()
    obs = of.mock_observations(fit, TRUTH, 10, (math.radians(-20), math.radians(20)), SIG, 3)
    c = _cfg()
    c.dt = 0.0
    with pytest.raises(nb.NBodyError) as e:
        nb.nbody_orbitfit_create(c, obs)
    assert e.value.code == nb.NBODY_EINVAL
    h = nb.nbody_orbitfit_create(_cfg(), obs)
    try:
        with pytest.raises(nb.NBodyError) as e:
            nb.nbody_orbitfit_eval(h, [TRUTH * np.array([1, -1, 1, 1, 1])])
        assert e.value.code == nb.NBODY_EINVAL
        with pytest.raises(nb.NBodyError) as e:
            nb.nbody_orbitfit_arc(h, TRUTH, max_pts=5)
        assert e.value.code == nb.NBODY_ESIZE
    finally:
        nb.nbody_orbitfit_destroy(h)

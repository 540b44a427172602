"""Pins of the orbit-fitting oracle (CPU only): unit conversions by their
definitions, observables of hand-placed points, proper motions and radial
velocity against differences of the angles and the distance along a
straight line, interpolation at the arc's nodes and midpoints, a zero
chi-square at the truth, and Gauss-Newton = half the Hessian there."""
import math

import numpy as np
import pytest

from oracle import orbitfit as of
from oracle import stream as ostream
from paper_2511_22468_gb300.configs import C1, G_KPC_MSUN_MYR

VSUN = np.array([12.9, 245.6, 7.78]) * of.KMS
TRUTH = np.array([1e12, 16.0, 6.8e10, 3.0, 0.28])
SIG = np.array([math.radians(0.1), 0.05, 0.05, 1.0])


def _fit():
    return of.OrbitFit(G_KPC_MSUN_MYR, C1.X0, C1.V0, C1.observer, VSUN,
                       (math.radians(-60), math.radians(60)), 0.5, 2000.0)


def test_unit_constants():
    assert of.MASYR == pytest.approx(180.0 / math.pi * 3600e3 / 1e6, rel=1e-15)
    year = 365.25 * 86400.0
    assert of.KMS == pytest.approx(1e6 * year / 3.0856775814913673e16, rel=1e-12)


def test_observables_of_hand_placed_points():
    fr = ostream.frame(C1.X0, C1.V0, C1.observer)
    e1, e2, n = fr
    xo, vo = np.array(C1.observer), np.array([0.01, -0.02, 0.003])
    D = 7.0
    q = of.observables(xo + D * e1, vo + 0.2 * e1, xo, vo, fr)[0]
    np.testing.assert_allclose(q, [0, 0, 0, 0, 0.2 / of.KMS], atol=1e-12)
    q = of.observables(xo + D * e1, vo + 0.2 * e2, xo, vo, fr)[0]
    np.testing.assert_allclose(q, [0, 0, 0.2 / D * of.MASYR, 0, 0], atol=1e-12)
    q = of.observables(xo + D * e2, vo - 0.2 * e1, xo, vo, fr)[0]     # phi1 = 90 deg
    np.testing.assert_allclose(q, [math.pi / 2, 0, 0.2 / D * of.MASYR, 0, 0], atol=1e-12)
    p = math.cos(math.radians(30)) * e1 + math.sin(math.radians(30)) * n
    q = of.observables(xo + D * p, vo + 0.2 * n, xo, vo, fr)[0]       # phi2 = 30 deg
    assert q[1] == pytest.approx(math.radians(30), abs=1e-13)
    assert q[3] == pytest.approx(0.2 * math.cos(math.radians(30)) / D * of.MASYR, rel=1e-12)


def test_proper_motions_are_angle_rates():
    """mu_phi1 cos phi2 = cos(phi2) dphi1/dt, mu_phi2 = dphi2/dt and
    v_h = dD/dt for relative motion along a straight line."""
    fr = ostream.frame(C1.X0, C1.V0, C1.observer)
    xo = np.array(C1.observer)
    rng = np.random.default_rng(0)
    for _ in range(5):
        x = xo + rng.normal(size=3) * 6
        w = rng.normal(size=3) * 0.2
        q = of.observables(x, w, xo, np.zeros(3), fr)[0]
        h = 1e-4
        qp = of.observables(x + w * h, w, xo, np.zeros(3), fr)[0]
        qm = of.observables(x - w * h, w, xo, np.zeros(3), fr)[0]
        dphi1 = (qp[0] - qm[0]) / (2 * h)
        dphi2 = (qp[1] - qm[1]) / (2 * h)
        dD = (np.linalg.norm(x + w * h - xo) - np.linalg.norm(x - w * h - xo)) / (2 * h)
        assert q[2] == pytest.approx(math.cos(q[1]) * dphi1 * of.MASYR, rel=1e-6, abs=1e-9)
        assert q[3] == pytest.approx(dphi2 * of.MASYR, rel=1e-6, abs=1e-9)
        assert q[4] == pytest.approx(dD / of.KMS, rel=1e-8)


def test_arc_and_interpolation():
    fit = _fit()
    A = fit.arc(TRUTH)
    assert len(A) > 100 and np.all(np.diff(A[:, 0]) > 0)
    k = len(A) // 3
    np.testing.assert_allclose(fit.model(TRUTH, A[[k, k + 1], 0]), A[[k, k + 1], 1:], rtol=1e-14)
    mid = fit.model(TRUTH, [0.5 * (A[k, 0] + A[k + 1, 0])])[0]
    np.testing.assert_allclose(mid, 0.5 * (A[k, 1:] + A[k + 1, 1:]), rtol=1e-12)
    # the progenitor sits at the frame's origin
    c = int(np.argmin(np.abs(A[:, 0])))
    assert abs(A[c, 0]) < 1e-14 and abs(A[c, 1]) < 1e-14


def test_zero_chi2_and_gauss_newton_at_the_truth():
    fit = _fit()
    obs = of.mock_observations(fit, TRUTH, 24, (math.radians(-40), math.radians(40)),
                               np.zeros(4), 0)
    assert fit.chi2(TRUTH, obs, SIG) == 0.0
    xi = np.log(TRUTH)
    f = lambda z: fit.chi2(np.exp(z), obs, SIG)         # noqa: E731
    H = of.fd_hessian(f, xi, h=1e-3)
    r = lambda z: fit.residuals(np.exp(z), obs, SIG)    # noqa: E731
    J = np.zeros((len(r(xi)), 5))
    for k in range(5):
        e = np.zeros(5)
        e[k] = 1e-6
        J[:, k] = (r(xi + e) - r(xi - e)) / 2e-6
    np.testing.assert_allclose(0.5 * H, J.T @ J, rtol=2e-3, atol=1e-6 * np.abs(J.T @ J).max())

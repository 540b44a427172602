"""Pins of the oracle's power-law bulge with exponential cut-off (the bulge of
MWPotential2014; CPU only).  The oracle integrates the density by
quadrature; the pins are the regularised incomplete gamma function of
scipy, the point-mass far field, -grad Phi, the Jacobian by differences,
Poisson's equation and the adjoint's bulge-mass gradient by differences."""
import dataclasses
import math

import numpy as np
import pytest
from scipy.special import gammainc

from oracle import core as o

G = 4.49850215e-12
MB, ALPHA, RC = 5e9, 1.8, 1.9
PH = o.Physics(G=G, ext=o.BULGE, bulge_M=MB, bulge_alpha=ALPHA, bulge_rc=RC)


@pytest.mark.parametrize("r", [0.01, 0.3, 1.0, 1.9, 4.0, 10.0])
def test_enclosed_mass_is_the_incomplete_gamma(orc, r):
    s = (3.0 - ALPHA) / 2.0
    assert o.bulge_mass(MB, ALPHA, RC, r) == pytest.approx(MB * gammainc(s, (r / RC) ** 2),
                                                           rel=1e-12)


def test_far_field_is_a_point_mass(orc):
    x = np.array([30.0, -20.0, 15.0])
    r = np.linalg.norm(x)
    np.testing.assert_allclose(o.ext_accel(PH, x), -G * MB * x / r ** 3, rtol=1e-13)


@pytest.mark.parametrize("p", [[0.3, 0.2, -0.1], [1.5, -0.7, 0.9], [4.0, 2.0, -3.0]])
def test_force_is_minus_grad_phi_and_jacobian(orc, p):
    p = np.array(p)
    a = o.ext_accel(PH, p)
    J = o.ext_jac(PH, p)
    for d in range(3):
        h = 1e-5 * np.linalg.norm(p)
        pp, pm = p.copy(), p.copy()
        pp[d] += h
        pm[d] -= h
        fd = -(o.ext_potential(PH, pp) - o.ext_potential(PH, pm)) / (2 * h)
        assert fd == pytest.approx(a[d], rel=1e-7, abs=1e-9 * np.abs(a).max())
        dA = (o.ext_accel(PH, pp) - o.ext_accel(PH, pm)) / (2 * h)
        np.testing.assert_allclose(dA, J[:, d], rtol=1e-6, atol=1e-7 * np.abs(J).max())


def test_poisson_equation(orc):
    """lap Phi = 4 pi G rho with rho(r) = rho_0 (r/r_1)^-alpha exp(-(r/r_c)^2),
    4 pi rho_0 r_1^alpha = 2 M_b / (r_c^(3-alpha) Gamma((3-alpha)/2))."""
    s = (3.0 - ALPHA) / 2.0
    for p in ([0.8, 0.3, -0.4], [2.0, 1.0, 1.5]):
        p = np.array(p)
        r = np.linalg.norm(p)
        rho4pi = 2.0 * MB / (RC ** (3.0 - ALPHA) * math.gamma(s)) * r ** -ALPHA * math.exp(-(r / RC) ** 2)
        h = 2e-3 * r
        lap = 0.0
        phi0 = o.ext_potential(PH, p)
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            lap += (o.ext_potential(PH, p + e) - 2 * phi0 + o.ext_potential(PH, p - e)) / h ** 2
        assert lap == pytest.approx(G * rho4pi, rel=2e-5)


def test_adjoint_bulge_mass_gradient_vs_fd(orc):
    rng = np.random.default_rng(9)
    n = 6
    x0 = rng.normal(size=(n, 3)) * 0.5 + np.array([2.0, 0.5, 0.3])
    v0 = rng.normal(size=(n, 3)) * 0.01 + np.array([0.0, 0.15, 0.02])
    m = np.full(n, 1e4)
    ph = dataclasses.replace(PH, eps=0.01, ext=o.BULGE | o.NFW | o.MN, nfw_M=1e12, nfw_rs=16.0,
                             mn_M=6.8e10, mn_a=3.0, mn_b=0.28)
    dt, steps = 0.5, 30
    wx, wv = rng.normal(size=(n, 3)), rng.normal(size=(n, 3))
    r = o.vjp(ph, x0, v0, m, dt, steps, wx, wv)

    def L(mb):
        xT, vT = o.integrate(dataclasses.replace(ph, bulge_M=mb), x0, v0, m, dt, steps)
        return np.sum(wx * xT) + np.sum(wv * vT)
    h = 1e-4 * MB
    d1 = (L(MB + h) - L(MB - h)) / (2 * h)
    d2 = (L(MB + h / 2) - L(MB - h / 2)) / h
    assert (4 * d2 - d1) / 3 == pytest.approx(r["bulge_M_bar"], rel=1e-6)
    # the position gradient through the bulge's Jacobian as well
    i, d = 2, 1
    def fx(e):
        xx = x0.copy()
        xx[i, d] += e
        xT, vT = o.integrate(ph, xx, v0, m, dt, steps)
        return np.sum(wx * xT) + np.sum(wv * vT)
    e = 1e-5
    assert (fx(e) - fx(-e)) / (2 * e) == pytest.approx(r["x0bar"][i, d], rel=1e-6)

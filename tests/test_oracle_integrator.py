"""Pins of the oracle's kick-drift-kick integrator and its discrete adjoint
(CPU only): closed forms, convergence order, reversibility, conservation
laws, and finite differences of the forward map."""
import json
import math
import os

import numpy as np
import pytest

from oracle import core as o
from paper_2511_22468_gb300.inputs import plummer_sphere

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "oracle_hand_values.json")))


def harm(omega2):
    return o.Physics(G=1.0, pair=False, ext=o.HARM, omega2=omega2)


def test_harmonic_one_step_map(orc):
    g = GOLD["harmonic_kdk_map"]
    M = np.array(g["map"])
    ph = harm(g["omega2"])
    for x0, v0 in ((1.0, 0.0), (0.0, 1.0), (0.3, -0.7)):
        x, v = o.integrate(ph, [[x0, 0, 0]], [[v0, 0, 0]], [1.0], g["h"], 1)
        np.testing.assert_allclose([x[0, 0], v[0, 0]], M @ [x0, v0], rtol=1e-15, atol=1e-16)
    # many steps equal the matrix power
    x, v = o.integrate(ph, [[0.3, 0, 0]], [[-0.7, 0, 0]], [1.0], g["h"], 50)
    np.testing.assert_allclose([x[0, 0], v[0, 0]],
                               np.linalg.matrix_power(M, 50) @ [0.3, -0.7], rtol=1e-12)


def test_harmonic_second_order_convergence(orc):
    """Error against cos/sin after fixed time T falls 4x per halving of h."""
    w2, T = 2.0, 3.0
    w = math.sqrt(w2)
    exact = math.cos(w * T) * 1.0 + math.sin(w * T) / w * 0.5
    errs = []
    for n in (100, 200, 400):
        x, v = o.integrate(harm(w2), [[1.0, 0, 0]], [[0.5, 0, 0]], [1.0], T / n, n)
        errs.append(abs(x[0, 0] - exact))
    assert errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)
    assert errs[1] / errs[2] == pytest.approx(4.0, rel=0.05)


def kepler_state(e=0.5, a=1.0):
    """Two bodies of mass 1/2 at apocentre, relative orbit with semi-major
    axis a and eccentricity e (G = 1, M = 1): period 2 pi a^1.5,
    energy -G m1 m2 / (2 a)."""
    ra = a * (1 + e)
    va = math.sqrt((1 - e) / (a * (1 + e)))
    x = np.array([[0.5 * ra, 0, 0], [-0.5 * ra, 0, 0]])
    v = np.array([[0, 0.5 * va, 0], [0, -0.5 * va, 0]])
    return x, v, np.array([0.5, 0.5])


def test_kepler_period_and_energy(orc):
    x0, v0, m = kepler_state()
    ph = o.Physics(G=1.0, eps=0.0)
    E0 = o.energy(ph, x0, v0, m)["E"]
    assert E0 == pytest.approx(-0.125, rel=1e-14)
    T = 2 * math.pi
    n = 2000
    x, v = o.integrate(ph, x0, v0, m, T / n, n)
    assert np.abs(x - x0).max() < 5e-3
    # bounded, non-drifting energy error over 20 orbits
    errs = []
    xs, vs = x0, v0
    for _ in range(20):
        xs, vs = o.integrate(ph, xs, vs, m, T / n, n)
        errs.append(abs(o.energy(ph, xs, vs, m)["E"] / E0 - 1))
    assert max(errs) < 1e-4
    assert errs[-1] < 3 * errs[0] + 1e-12


def test_time_reversibility(orc):
    x0, v0, m = plummer_sphere(64, 11, 1.0, 1.0, 1.0)
    ph = o.Physics(G=1.0, eps=0.05, ext=o.HARM, omega2=0.3)
    x, v = o.integrate(ph, x0, v0, m, 1e-3, 200)
    xb, vb = o.integrate(ph, x, -v, m, 1e-3, 200)
    assert np.abs(xb - x0).max() < 1e-12 * np.abs(x0).max()
    assert np.abs(-vb - v0).max() < 1e-11 * np.abs(v0).max()


def test_momentum_conserved_without_external(orc):
    x0, v0, m = plummer_sphere(128, 12, 1.0, 1.0, 1.0)
    m = m * np.linspace(0.5, 1.5, 128)
    ph = o.Physics(G=1.0, eps=0.01)
    P0 = o.energy(ph, x0, v0, m)["P"]
    x, v = o.integrate(ph, x0, v0, m, 1e-3, 300)
    P = o.energy(ph, x, v, m)["P"]
    assert np.abs(P - P0).max() < 1e-15


def test_plummer_energy_closed_form_and_bounded_error(orc):
    """The sampled sphere's energy is near -3 pi G M^2/(64 a) (unsoftened,
    N -> infinity) and its KDK energy error stays small over the Plummer
    workload's 1000 steps (N = 1024, eps = 0.01, dt = 1e-3)."""
    x0, v0, m = plummer_sphere(1024, 0, 1.0, 1.0, 1.0)
    ph = o.Physics(G=1.0, eps=0.01)
    e0 = o.energy(ph, x0, v0, m)
    assert e0["E"] == pytest.approx(-3 * math.pi / 64, rel=0.08)
    assert 2 * e0["K"] / -e0["W_pair"] == pytest.approx(1.0, abs=0.1)
    x, v = o.integrate(ph, x0, v0, m, 1e-3, 1000)
    e1 = o.energy(ph, x, v, m)
    assert abs(e1["E"] / e0["E"] - 1) < 2e-4


# ------------------------------------------------------------------ adjoint --
def _loss(ph, x0, v0, m, dt, n, wx, wv):
    x, v = o.integrate(ph, x0, v0, m, dt, n)
    return np.sum(wx * x) + np.sum(wv * v)


def test_adjoint_harmonic_closed_form(orc):
    """For the linear map z_n = M(h)^n z_0: dL/dz_0 = (M^n)^T w, and
    dL/dh = w . d(M^n)/dh z_0 with M(h) from the hand-derived map."""
    w2, h, n = 4.0, 0.1, 30
    z0 = np.array([0.3, -0.7])
    w = np.array([1.3, 0.4])

    def Mh(hh):
        c = 1 - hh * hh * w2 / 2
        return np.array([[c, hh], [-hh * w2 * (1 - hh * hh * w2 / 4), c]])

    def Mdh(hh):
        return np.array([[-hh * w2, 1.0],
                         [-w2 * (1 - 3 * hh * hh * w2 / 4), -hh * w2]])

    Mn = np.linalg.matrix_power(Mh(h), n)
    dMn = sum(np.linalg.matrix_power(Mh(h), n - 1 - k) @ Mdh(h) @ np.linalg.matrix_power(Mh(h), k)
              for k in range(n))
    r = o.vjp(harm(w2), [[z0[0], 0, 0]], [[z0[1], 0, 0]], [1.0], h, n,
              [[w[0], 0, 0]], [[w[1], 0, 0]])
    g = Mn.T @ w
    assert r["x0bar"][0, 0] == pytest.approx(g[0], rel=1e-12)
    assert r["v0bar"][0, 0] == pytest.approx(g[1], rel=1e-12)
    assert r["dt_bar"] == pytest.approx(w @ dMn @ z0, rel=1e-11)


@pytest.mark.parametrize("ext", [0, o.NFW | o.MN])
def test_adjoint_vs_central_fd(orc, ext):
    """Every gradient of the oracle adjoint against central differences of
    the forward map (Richardson-extrapolated)."""
    rng = np.random.default_rng(5)
    n_p = 24
    x0, v0, m = plummer_sphere(n_p, 21, 1.0, 1.0, 1.0)
    m = m * rng.uniform(0.5, 1.5, n_p)
    if ext:
        # place the cluster on an orbit in a scaled NFW + MN field
        x0 = x0 + np.array([4.0, 1.0, 0.5])
        v0 = v0 + np.array([0.0, 0.4, 0.1])
    ph = o.Physics(G=1.0, eps=0.1, ext=ext, nfw_M=2.0, nfw_rs=3.0, mn_M=1.0,
                   mn_a=1.0, mn_b=0.3)
    dt, n = 0.01, 40
    wx = rng.normal(size=(n_p, 3))
    wv = rng.normal(size=(n_p, 3))
    r = o.vjp(ph, x0, v0, m, dt, n, wx, wv)

    def fd(f, h):
        d1 = (f(h) - f(-h)) / (2 * h)
        d2 = (f(h / 2) - f(-h / 2)) / h
        return (4 * d2 - d1) / 3

    L = lambda **kw: _loss(kw.get("ph", ph), kw.get("x0", x0), kw.get("v0", v0),
                           kw.get("m", m), kw.get("dt", dt), n, wx, wv)
    for (i, d) in ((0, 0), (7, 2), (23, 1)):
        def fx(h):
            xx = x0.copy()
            xx[i, d] += h
            return L(x0=xx)

        def fv(h):
            vv = v0.copy()
            vv[i, d] += h
            return L(v0=vv)
        assert fd(fx, 1e-4) == pytest.approx(r["x0bar"][i, d], rel=1e-6, abs=1e-9)
        assert fd(fv, 1e-4) == pytest.approx(r["v0bar"][i, d], rel=1e-6, abs=1e-9)
    for j in (2, 19):
        def fm(h):
            mm = m.copy()
            mm[j] += h
            return L(m=mm)
        assert fd(fm, 1e-4) == pytest.approx(r["mbar"][j], rel=1e-6, abs=1e-9)
    assert fd(lambda h: L(dt=dt + h), 1e-5) == pytest.approx(r["dt_bar"], rel=1e-6)
    if ext:
        import dataclasses
        fn = lambda h: L(ph=dataclasses.replace(ph, nfw_M=ph.nfw_M + h))
        fm_ = lambda h: L(ph=dataclasses.replace(ph, mn_M=ph.mn_M + h))
        assert fd(fn, 1e-4) == pytest.approx(r["nfw_M_bar"], rel=1e-6)
        assert fd(fm_, 1e-4) == pytest.approx(r["mn_M_bar"], rel=1e-6)
        # shape parameters of the halo and the disk
        for key, name in (("nfw_rs", "nfw_rs_bar"), ("mn_a", "mn_a_bar"),
                          ("mn_b", "mn_b_bar")):
            f = lambda h, key=key: L(ph=dataclasses.replace(ph, **{key: getattr(ph, key) + h}))
            assert fd(f, 1e-4) == pytest.approx(r[name], rel=1e-6)


def test_adjoint_dot_product(orc):
    """<J delta, w> = <delta, J^T w> with J delta from central differences."""
    rng = np.random.default_rng(6)
    x0, v0, m = plummer_sphere(32, 22, 1.0, 1.0, 1.0)
    ph = o.Physics(G=1.0, eps=0.05)
    dt, n = 0.01, 25
    dx = rng.normal(size=x0.shape)
    dv = rng.normal(size=v0.shape)
    wx = rng.normal(size=x0.shape)
    wv = rng.normal(size=v0.shape)
    h = 1e-5
    xp, vp = o.integrate(ph, x0 + h * dx, v0 + h * dv, m, dt, n)
    xm, vm = o.integrate(ph, x0 - h * dx, v0 - h * dv, m, dt, n)
    jvp = (np.sum(wx * (xp - xm)) + np.sum(wv * (vp - vm))) / (2 * h)
    r = o.vjp(ph, x0, v0, m, dt, n, wx, wv, want_mbar=False)
    vjp = np.sum(dx * r["x0bar"]) + np.sum(dv * r["v0bar"])
    assert vjp == pytest.approx(jvp, rel=1e-7)


def test_mass_scale_gradient_identity(orc):
    """sum_j m_j dL/dm_j equals the kick-weighted sum of lam . a_pair over
    the trajectory: the shortcut the GPU adjoint uses for the progenitor
    mass, checked against the oracle's per-particle mass gradient."""
    x0, v0, m = plummer_sphere(20, 23, 1.0, 1.0, 1.0)
    ph = o.Physics(G=1.0, eps=0.05)
    rng = np.random.default_rng(7)
    wx = rng.normal(size=x0.shape)
    dt, n = 0.02, 15
    r = o.vjp(ph, x0, v0, m, dt, n, wx, np.zeros_like(wx))
    # scaling every mass by (1 + s): central difference in s
    s = 1e-5
    Lp = _loss(ph, x0, v0, m * (1 + s), dt, n, wx, 0 * wx)
    Lm = _loss(ph, x0, v0, m * (1 - s), dt, n, wx, 0 * wx)
    assert np.dot(m, r["mbar"]) == pytest.approx((Lp - Lm) / (2 * s), rel=1e-7)

"""Pins of the oracle's force model against hand values, closed forms,
invariants and finite differences (CPU only)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import core as o
from paper_2511_22468_gb300.inputs import plummer_sphere

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "oracle_hand_values.json")))


# ---------------------------------------------------------------- pair sum --
def test_pair_hand_345(orc):
    g = GOLD["pair_345"]
    x, m = np.array(g["x"], float), np.array(g["m"])
    a = o.pair_accel(x, m, g["G"], g["eps"])
    np.testing.assert_allclose(a, g["acc"], rtol=0, atol=1e-15)
    assert o.pair_potential(x, m, g["G"], g["eps"]) == pytest.approx(g["W"], abs=1e-15)
    gv = o.pair_vjp(x, m, g["G"], g["eps"], np.array(g["vjp_lam"], float))
    np.testing.assert_allclose(gv, g["vjp_g"], rtol=0, atol=1e-16)
    mv = o.pair_mass_vjp(x, g["G"], g["eps"], np.array(g["mass_vjp_lam"], float))
    np.testing.assert_allclose(mv, g["mass_vjp"], rtol=0, atol=1e-16)


def test_pair_equilateral(orc):
    g = GOLD["equilateral"]
    x, m = np.array(g["x"]), np.array(g["m"])
    a = o.pair_accel(x, m, g["G"], g["eps"])
    c = x.mean(axis=0)
    for i in range(3):
        assert np.linalg.norm(a[i]) == pytest.approx(g["acc_norm"], rel=1e-14)
        d = (c - x[i]) / np.linalg.norm(c - x[i])
        assert np.dot(a[i], d) == pytest.approx(g["acc_norm"], rel=1e-14)
    assert o.pair_potential(x, m, g["G"], g["eps"]) == pytest.approx(g["W"], rel=1e-14)


def test_pair_third_law_and_rows(orc):
    x, v, m = plummer_sphere(300, 5, 1.0, 1.0, 1.0)
    m = m * np.linspace(0.5, 1.5, 300)  # unequal masses
    a = o.pair_accel(x, m, 1.0, 0.02)
    P = (m[:, None] * a).sum(axis=0)
    assert np.abs(P).max() < 1e-14 * np.abs(m[:, None] * a).sum()
    rows = np.array([7, 0, 299, 150])
    np.testing.assert_array_equal(o.pair_accel(x, m, 1.0, 0.02, rows=rows), a[rows])


def test_pair_accel_is_minus_grad_potential(orc):
    x, v, m = plummer_sphere(64, 3, 1.0, 1.0, 1.0)
    a = o.pair_accel(x, m, 1.0, 0.05)
    h = 1e-5
    for i in (0, 17, 63):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            fd = -(o.pair_potential(xp, m, 1.0, 0.05) - o.pair_potential(xm, m, 1.0, 0.05)) / (2 * h)
            assert fd / m[i] == pytest.approx(a[i, d], rel=1e-6, abs=1e-9)


def test_pair_vjp_matches_fd_jacobian(orc):
    rng = np.random.default_rng(0)
    x, v, m = plummer_sphere(40, 4, 1.0, 1.0, 1.0)
    m = m * rng.uniform(0.5, 2.0, 40)
    lam = rng.normal(size=(40, 3))
    eps = 0.03
    g = o.pair_vjp(x, m, 1.0, eps, lam)
    h = 1e-6
    for k in (0, 11, 39):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[k, d] += h
            xm[k, d] -= h
            dA = (o.pair_accel(xp, m, 1.0, eps) - o.pair_accel(xm, m, 1.0, eps)) / (2 * h)
            assert np.sum(dA * lam) == pytest.approx(g[k, d], rel=1e-6, abs=1e-8)
    # mass gradient: Euler's theorem, a is homogeneous of degree 1 in m
    mb = o.pair_mass_vjp(x, 1.0, eps, lam)
    assert np.dot(m, mb) == pytest.approx(np.sum(lam * o.pair_accel(x, m, 1.0, eps)), rel=1e-12)
    for j in (3, 30):
        mp, mm = m.copy(), m.copy()
        mp[j] += 1e-6
        mm[j] -= 1e-6
        fd = np.sum(lam * (o.pair_accel(x, mp, 1.0, eps) - o.pair_accel(x, mm, 1.0, eps))) / 2e-6
        assert fd == pytest.approx(mb[j], rel=1e-6)
    # row selections give the rows of the full products
    rows = np.array([39, 0, 17])
    assert np.array_equal(o.pair_mass_vjp(x, 1.0, eps, lam, rows=rows), mb[rows])
    assert np.array_equal(o.pair_vjp(x, m, 1.0, eps, lam, rows=rows), g[rows])


def test_pair_mean_field_plummer(orc):
    """Weak pin: a sampled Plummer sphere's pair force follows the model's
    mean field -G M r/(r^2 + a^2)^(3/2) within Poisson noise."""
    x, v, m = plummer_sphere(20000, 9, 1.0, 1.0, 1.0)
    r = np.linalg.norm(x, axis=1)
    rows = np.where((r > 0.5) & (r < 2.0))[0][:200]
    a = o.pair_accel(x, m, 1.0, 0.0, rows=rows)
    model = -x[rows] / (r[rows] ** 2 + 1.0)[:, None] ** 1.5
    rad = np.sum(a * x[rows], axis=1) / r[rows]
    rad_model = np.sum(model * x[rows], axis=1) / r[rows]
    assert np.median(np.abs(rad / rad_model - 1.0)) < 0.05
    assert abs(np.mean(rad / rad_model) - 1.0) < 0.03


# --------------------------------------------------------------- external --
def test_nfw_hand_values(orc):
    g = GOLD["nfw_at_rs"]
    ph = o.Physics(G=1.0, pair=False, ext=o.NFW, nfw_M=1.0, nfw_rs=g["rs"])
    assert o.ext_potential(ph, g["x"]) == pytest.approx(g["phi"], rel=1e-14)
    a = o.ext_accel(ph, g["x"])
    assert a[0] == pytest.approx(g["acc_x"], rel=1e-13)
    assert abs(a[1]) + abs(a[2]) == 0.0
    assert np.trace(o.ext_jac(ph, g["x"])) == pytest.approx(g["trace_jac"], rel=1e-12)


def test_nfw_enclosed_mass_and_laplacian(orc):
    """|a| = G M(<r)/r^2 with M(<r) = M [ln(1+x) - x/(1+x)] (Gauss), and
    trace(da/dx) = -4 pi G rho for rho = M / (4 pi r (r + r_s)^2)."""
    G, M, rs = 4.5e-12, 1e12, 16.0
    ph = o.Physics(G=G, pair=False, ext=o.NFW, nfw_M=M, nfw_rs=rs)
    rng = np.random.default_rng(1)
    for r in (0.3, 2.0, 14.0, 16.0, 60.0, 400.0):
        u = rng.normal(size=3)
        p = r * u / np.linalg.norm(u)
        q = r / rs
        menc = M * (math.log(1 + q) - q / (1 + q))
        a = o.ext_accel(ph, p)
        assert np.linalg.norm(a) == pytest.approx(G * menc / r ** 2, rel=1e-11)
        assert np.dot(a, p) < 0
        rho = M / (4 * math.pi * r * (r + rs) ** 2)
        assert np.trace(o.ext_jac(ph, p)) == pytest.approx(-4 * math.pi * G * rho, rel=1e-9)


def test_nfw_series_branch_is_continuous(orc):
    ph = o.Physics(G=1.0, pair=False, ext=o.NFW, nfw_M=1.0, nfw_rs=16.0)
    r0 = 16.0 * 1e-4
    lo = o.ext_accel(ph, [r0 * (1 - 1e-9), 0, 0])
    hi = o.ext_accel(ph, [r0 * (1 + 1e-9), 0, 0])
    assert lo[0] == pytest.approx(hi[0], rel=1e-8)
    # centre limit: |a| -> G M / (2 r_s^2)
    a = o.ext_accel(ph, [1e-9, 0, 0])
    assert -a[0] == pytest.approx(1.0 / (2 * 16.0 ** 2), rel=1e-6)


def test_mn_hand_values(orc):
    for c in GOLD["mn_cases"]["cases"]:
        ph = o.Physics(G=1.0, pair=False, ext=o.MN, mn_M=1.0, mn_a=c["a"], mn_b=c["b"])
        assert o.ext_potential(ph, c["x"]) == pytest.approx(c["phi"], rel=1e-14)
        np.testing.assert_allclose(o.ext_accel(ph, c["x"]), c["acc"], rtol=1e-14, atol=1e-17)


def test_mn_reductions_and_laplacian(orc):
    """a = 0 gives a Plummer sphere of scale b; far away a point mass; the
    trace of da/dx is -4 pi G rho with the Miyamoto-Nagai density
    rho = b^2 M [a R^2 + (a + 3B)(a + B)^2] / (4 pi S^5 B^3)."""
    rng = np.random.default_rng(2)
    ph = o.Physics(G=1.0, pair=False, ext=o.MN, mn_M=1.0, mn_a=0.0, mn_b=0.7)
    for _ in range(5):
        p = rng.normal(size=3)
        r2 = p @ p
        np.testing.assert_allclose(o.ext_accel(ph, p), -p / (r2 + 0.49) ** 1.5, rtol=1e-13)
    ph = o.Physics(G=1.0, pair=False, ext=o.MN, mn_M=1.0, mn_a=3.0, mn_b=0.28)
    p = np.array([3e4, -1e4, 2e4])
    assert o.ext_potential(ph, p) == pytest.approx(-1 / np.linalg.norm(p), rel=3e-4)
    for _ in range(6):
        p = rng.normal(size=3) * np.array([6, 6, 2])
        R2 = p[0] ** 2 + p[1] ** 2
        B = math.sqrt(p[2] ** 2 + 0.28 ** 2)
        S2 = R2 + (3 + B) ** 2
        rho = 0.28 ** 2 * (3 * R2 + (3 + 3 * B) * (3 + B) ** 2) / (4 * math.pi * S2 ** 2.5 * B ** 3)
        assert np.trace(o.ext_jac(ph, p)) == pytest.approx(-4 * math.pi * rho, rel=1e-9)


@pytest.mark.parametrize("ext", [o.NFW, o.MN, o.NFW | o.MN])
def test_ext_accel_and_jacobian_vs_fd(orc, ext):
    ph = o.Physics(G=4.5e-12, pair=False, ext=ext, nfw_M=1e12, nfw_rs=16.0,
                   mn_M=6.8e10, mn_a=3.0, mn_b=0.28)
    rng = np.random.default_rng(3)
    for _ in range(6):
        p = rng.normal(size=3) * np.array([10, 10, 3])
        a = o.ext_accel(ph, p)
        J = o.ext_jac(ph, p)
        np.testing.assert_allclose(J, J.T, rtol=1e-12, atol=1e-12 * np.abs(J).max())
        for d in range(3):
            h = 1e-5 * max(1.0, abs(p[d]))
            pp, pm = p.copy(), p.copy()
            pp[d] += h
            pm[d] -= h
            fd = -(o.ext_potential(ph, pp) - o.ext_potential(ph, pm)) / (2 * h)
            assert fd == pytest.approx(a[d], rel=1e-7, abs=1e-9 * np.abs(a).max())
            dA = (o.ext_accel(ph, pp) - o.ext_accel(ph, pm)) / (2 * h)
            np.testing.assert_allclose(dA, J[:, d], rtol=1e-6, atol=1e-7 * np.abs(J).max())
    parts = o.ext_accel_parts(ph, [5.0, 1.0, 2.0])
    np.testing.assert_allclose(parts.sum(axis=0), o.ext_accel(ph, [5.0, 1.0, 2.0]), rtol=1e-15)


def test_circular_speed_of_stream_potential(orc):
    """Sanity of units and of the NFW-mass reading: v_c at 14 kpc in the
    workload's halo + disk is about 230-270 km/s."""
    from paper_2511_22468_gb300.configs import C1
    p = C1.pot
    ph = o.Physics(G=C1.G, pair=False, ext=o.NFW | o.MN, nfw_M=p.nfw_M,
                   nfw_rs=p.nfw_rs, mn_M=p.mn_M, mn_a=p.mn_a, mn_b=p.mn_b)
    a = o.ext_accel(ph, [14.0, 0.0, 0.0])
    vc_kms = math.sqrt(-a[0] * 14.0) / 1.0227122e-3
    assert 200.0 < vc_kms < 290.0

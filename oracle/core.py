"""ctypes wrapper of the FP64 C oracle (TEST INFRASTRUCTURE ONLY).

Arrays are numpy float64, positions and velocities shaped (n, 3).  See
``nbody_oracle.c`` for the definitions each routine writes out:
softened pair gravity (paper Sec. 1), NFW + Miyamoto-Nagai potentials and the
Velocity-Verlet integrator (Sec. 2.2.1), reverse-mode gradients (Sec. 2).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from .build import build_oracle

NFW = 1
MN = 2
HARM = 4
BULGE = 8


class OrcParams(C.Structure):
    _fields_ = [("G", C.c_double), ("eps", C.c_double), ("pair", C.c_int32),
                ("ext", C.c_uint32), ("nfw_M", C.c_double),
                ("nfw_rs", C.c_double), ("mn_M", C.c_double),
                ("mn_a", C.c_double), ("mn_b", C.c_double),
                ("omega2", C.c_double), ("bulge_M", C.c_double),
                ("bulge_alpha", C.c_double), ("bulge_rc", C.c_double)]


@dataclass
class Physics:
    """Force model: softened pair sum plus optional external components."""
    G: float = 1.0
    eps: float = 0.0
    pair: bool = True
    ext: int = 0
    nfw_M: float = 0.0
    nfw_rs: float = 1.0
    mn_M: float = 0.0
    mn_a: float = 0.0
    mn_b: float = 0.0
    omega2: float = 0.0
    bulge_M: float = 0.0
    bulge_alpha: float = 1.8
    bulge_rc: float = 1.9

    def c(self) -> OrcParams:
        return OrcParams(self.G, self.eps, int(self.pair), self.ext,
                         self.nfw_M, self.nfw_rs, self.mn_M, self.mn_a,
                         self.mn_b, self.omega2, self.bulge_M, self.bulge_alpha,
                         self.bulge_rc)


_lib = None
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build_oracle())
        P = C.POINTER(OrcParams)
        L.orc_pair_accel.argtypes = [C.c_int64, _D, _D, C.c_double, C.c_double,
                                     _I64, C.c_int64, _D]
        L.orc_pair_potential.argtypes = [C.c_int64, _D, _D, C.c_double, C.c_double]
        L.orc_pair_potential.restype = C.c_double
        L.orc_pair_vjp.argtypes = [C.c_int64, _D, _D, C.c_double, C.c_double, _D,
                                   _I64, C.c_int64, _D]
        L.orc_pair_mass_vjp.argtypes = [C.c_int64, _D, C.c_double, C.c_double,
                                        _D, _I64, C.c_int64, _D]
        L.orc_ext_accel_parts.argtypes = [P, _D, _D]
        L.orc_ext_accel.argtypes = [P, _D, _D]
        L.orc_ext_potential.argtypes = [P, _D]
        L.orc_ext_potential.restype = C.c_double
        L.orc_ext_jac.argtypes = [P, _D, _D]
        L.orc_accel.argtypes = [P, C.c_int64, _D, _D, _D]
        L.orc_integrate.argtypes = [P, C.c_int64, _D, _D, _D, C.c_double,
                                    C.c_int64, _D, _D]
        L.orc_integrate.restype = C.c_int
        L.orc_energy.argtypes = [P, C.c_int64, _D, _D, _D, _D]
        L.orc_vjp.argtypes = [P, C.c_int64, _D, _D, _D, C.c_double, C.c_int64,
                              _D, _D, _D, _D, _D, _D]
        L.orc_vjp.restype = C.c_int
        L.orc_bulge_mass.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double]
        L.orc_bulge_mass.restype = C.c_double
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def pair_accel(x, m, G, eps, rows=None):
    """Softened pair acceleration of rows (all particles when rows is None)."""
    x = _f64(x, (-1, 3))
    m = _f64(m, (-1,))
    n = x.shape[0]
    if rows is None:
        nr, rp = n, None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nr, rp = rows.shape[0], rows.ctypes.data_as(_I64)
    out = np.zeros((nr, 3))
    lib().orc_pair_accel(n, _d(x), _d(m), G, eps, rp, nr, _d(out))
    return out


def pair_potential(x, m, G, eps):
    x = _f64(x, (-1, 3))
    m = _f64(m, (-1,))
    return lib().orc_pair_potential(x.shape[0], _d(x), _d(m), G, eps)


def pair_vjp(x, m, G, eps, lam, rows=None):
    """g_k = sum_i (d a_i / d x_k)^T lam_i for rows k."""
    x = _f64(x, (-1, 3))
    m = _f64(m, (-1,))
    lam = _f64(lam, (-1, 3))
    n = x.shape[0]
    if rows is None:
        nr, rp = n, None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nr, rp = rows.shape[0], rows.ctypes.data_as(_I64)
    out = np.zeros((nr, 3))
    lib().orc_pair_vjp(n, _d(x), _d(m), G, eps, _d(lam), rp, nr, _d(out))
    return out


def pair_mass_vjp(x, G, eps, lam, rows=None):
    """mbar_j = sum_i lam_i . d a_i / d m_j for rows j (all when None)."""
    x = _f64(x, (-1, 3))
    lam = _f64(lam, (-1, 3))
    n = x.shape[0]
    if rows is None:
        nr, rp = n, None
    else:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nr, rp = rows.shape[0], rows.ctypes.data_as(_I64)
    out = np.zeros(nr)
    lib().orc_pair_mass_vjp(n, _d(x), G, eps, _d(lam), rp, nr, _d(out))
    return out


def ext_accel_parts(ph: Physics, x3):
    """(NFW, MN, harmonic, bulge) accelerations at one point, each shape (3,)."""
    x3 = _f64(x3, (3,))
    out = np.zeros(12)
    p = ph.c()
    lib().orc_ext_accel_parts(C.byref(p), _d(x3), _d(out))
    return out.reshape(4, 3)


def ext_accel(ph: Physics, x3):
    x3 = _f64(x3, (3,))
    out = np.zeros(3)
    p = ph.c()
    lib().orc_ext_accel(C.byref(p), _d(x3), _d(out))
    return out


def ext_potential(ph: Physics, x3):
    x3 = _f64(x3, (3,))
    p = ph.c()
    return lib().orc_ext_potential(C.byref(p), _d(x3))


def ext_jac(ph: Physics, x3):
    """J[a, b] = d a_a / d x_b of the external acceleration at one point."""
    x3 = _f64(x3, (3,))
    out = np.zeros(9)
    p = ph.c()
    lib().orc_ext_jac(C.byref(p), _d(x3), _d(out))
    return out.reshape(3, 3)


def accel(ph: Physics, x, m):
    x = _f64(x, (-1, 3))
    m = _f64(m, (-1,))
    out = np.zeros_like(x)
    p = ph.c()
    lib().orc_accel(C.byref(p), x.shape[0], _d(x), _d(m), _d(out))
    return out


def integrate(ph: Physics, x0, v0, m, dt, nsteps, traj=False):
    """Kick-drift-kick for nsteps; returns (x, v) or (x, v, X, VH) with the
    positions x_0..x_n and half-step velocities when traj is True."""
    x = _f64(x0, (-1, 3)).copy()
    v = _f64(v0, (-1, 3)).copy()
    m = _f64(m, (-1,))
    n = x.shape[0]
    X = np.zeros((nsteps + 1, n, 3)) if traj else None
    VH = np.zeros((max(nsteps, 1), n, 3)) if traj else None
    p = ph.c()
    rc = lib().orc_integrate(C.byref(p), n, _d(x), _d(v), _d(m), dt, nsteps,
                             _d(X), _d(VH))
    if rc:
        raise MemoryError("oracle integrate failed (%d)" % rc)
    if traj:
        return x, v, X, VH[:nsteps]
    return x, v


def energy(ph: Physics, x, v, m):
    """dict(K, W_pair, W_ext, E, P)."""
    x = _f64(x, (-1, 3))
    v = _f64(v, (-1, 3))
    m = _f64(m, (-1,))
    out = np.zeros(6)
    p = ph.c()
    lib().orc_energy(C.byref(p), x.shape[0], _d(x), _d(v), _d(m), _d(out))
    return dict(K=out[0], W_pair=out[1], W_ext=out[2],
                E=out[0] + out[1] + out[2], P=out[3:6].copy())


def vjp(ph: Physics, x0, v0, m, dt, nsteps, xbar, vbar, want_mbar=True):
    """Reverse-mode gradient of L(x_T, v_T) through integrate().

    Returns dict(x0bar, v0bar, mbar, dt_bar, nfw_M_bar, mn_M_bar, nfw_rs_bar,
    mn_a_bar, mn_b_bar, bulge_M_bar)."""
    x0 = _f64(x0, (-1, 3))
    v0 = _f64(v0, (-1, 3))
    m = _f64(m, (-1,))
    xbar = _f64(xbar, (-1, 3))
    vbar = _f64(vbar, (-1, 3))
    n = x0.shape[0]
    x0b = np.zeros_like(x0)
    v0b = np.zeros_like(v0)
    mb = np.zeros(n) if want_mbar else None
    pb = np.zeros(7)
    p = ph.c()
    rc = lib().orc_vjp(C.byref(p), n, _d(x0), _d(v0), _d(m), dt, nsteps,
                       _d(xbar), _d(vbar), _d(x0b), _d(v0b), _d(mb), _d(pb))
    if rc:
        raise MemoryError("oracle vjp failed (%d)" % rc)
    return dict(x0bar=x0b, v0bar=v0b, mbar=mb, dt_bar=pb[0], nfw_M_bar=pb[1],
                mn_M_bar=pb[2], nfw_rs_bar=pb[3], mn_a_bar=pb[4], mn_b_bar=pb[5],
                bulge_M_bar=pb[6])


def bulge_mass(M_b, alpha, r_c, r):
    """Enclosed mass of the power-law bulge (quadrature of its density)."""
    return lib().orc_bulge_mass(M_b, alpha, r_c, r)

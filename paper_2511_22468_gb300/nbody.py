"""Thin Python binding of libnbody (include/nbody.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  Functions carry the C names; arrays are torch
tensors (device or pinned/pageable host) or numpy arrays, FP64, laid out
structure-of-arrays: positions and velocities (3, n), masses (n,).
The library is loaded on first use and a missing library raises, so no
call can silently fall back to another implementation.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
# NBODY_LIBRARY selects another build of the same library (e.g. one built
# with different tile sizes); the default is the in-tree build.
LIB_PATH = os.environ.get("NBODY_LIBRARY", os.path.join(PKG, "_build", "libnbody.so"))

NBODY_OK = 0
NBODY_EINVAL = -1
NBODY_ENOMEM = -2
NBODY_ECUDA = -3
NBODY_ETIMEOUT = -4
NBODY_ENAN = -5
NBODY_ESTATE = -6
NBODY_ENODEV = -7
NBODY_ESIZE = -8
NBODY_NOALLOC_MAX_N = 32768

NBODY_EXT_NFW = 1
NBODY_EXT_MN = 2
NBODY_EXT_BULGE = 4
NBODY_CENTER_FIXED = 0
NBODY_CENTER_GUIDE = 1
NBODY_TAPE_KEEP_LAST = 0
NBODY_TAPE_LEAN = 1

EXPORTED = ("nbody_create", "nbody_destroy", "nbody_set_params",
            "nbody_set_state", "nbody_get_state", "nbody_step",
            "nbody_integrate", "nbody_vjp", "nbody_energy", "nbody_momentum",
            "nbody_get_status", "nbody_strerror", "nbody_launch_count",
            "nbody_pair_accel", "nbody_set_timing", "nbody_kernel_times",
            "nbody_pair_accel_noalloc", "nbody_stream_create",
            "nbody_stream_set_target", "nbody_stream_forward", "nbody_stream_grad",
            "nbody_stream_destroy", "nbody_stream_initial_state", "nbody_stream_head", "nbody_create_batch",
            "nbody_vjp_batch", "nbody_autotune",
            "nbody_set_tuning", "nbody_get_tuning", "nbody_mlp_create",
            "nbody_mlp_num_params", "nbody_mlp_set_params", "nbody_mlp_get_params",
            "nbody_mlp_forward", "nbody_mlp_loss_grad", "nbody_mlp_adam_step",
            "nbody_mlp_destroy", "nbody_mlp_invert", "nbody_mlp_get_status", "nbody_set_pair_shape",
            "nbody_set_pair_finish", "nbody_get_pair_shape", "nbody_set_pair_tile",
            "nbody_get_pair_tile", "nbody_peaks", "nbody_autotune_pair",
            "nbody_potential_grad", "nbody_mmd_create", "nbody_mmd_eval",
            "nbody_mmd_eval_batch", "nbody_mmd_eval_cross", "nbody_mmd_target_stats",
            "nbody_mmd_destroy",
            "nbody_stream_set_target_cloud", "nbody_stream_initial_states",
            "nbody_ext_accel", "nbody_stream_autotune", "nbody_stream_get_pair_shape", "nbody_orbitfit_create", "nbody_orbitfit_eval",
            "nbody_orbitfit_lm", "nbody_orbitfit_fisher", "nbody_orbitfit_arc",
            "nbody_orbitfit_destroy", "nbody_stream_batch_create",
            "nbody_stream_batch_loss_grad", "nbody_stream_batch_grad_parts",
            "nbody_stream_batch_destroy")

NBODY_NTUNE = 8

NBODY_KCLASS = ("pair", "vjp", "update", "adjoint", "field")


class nbody_params(C.Structure):
    _fields_ = [("G", C.c_double), ("eps", C.c_double), ("dt", C.c_double),
                ("checkpoint_every", C.c_int64), ("ext_flags", C.c_uint32),
                ("center_mode", C.c_uint32), ("tape_mode", C.c_uint32),
                ("reserved", C.c_uint32), ("nfw_M", C.c_double),
                ("nfw_rs", C.c_double), ("mn_M", C.c_double),
                ("mn_a", C.c_double), ("mn_b", C.c_double),
                ("center", C.c_double * 3), ("center_vel", C.c_double * 3),
                ("bulge_M", C.c_double), ("bulge_alpha", C.c_double),
                ("bulge_rc", C.c_double)]


class nbody_orbitfit_cfg(C.Structure):
    _fields_ = [("G", C.c_double), ("X0", C.c_double * 3), ("V0", C.c_double * 3),
                ("observer", C.c_double * 3), ("observer_vel", C.c_double * 3),
                ("phi1_lo", C.c_double), ("phi1_hi", C.c_double), ("dt", C.c_double),
                ("t_max", C.c_double), ("sigma", C.c_double * 4)]


class nbody_stream_cfg(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_steps", C.c_int64),
                ("checkpoint_every", C.c_int64), ("G", C.c_double),
                ("eps", C.c_double), ("a_prog", C.c_double), ("nfw_rs", C.c_double),
                ("mn_a", C.c_double), ("mn_b", C.c_double),
                ("X0", C.c_double * 3), ("V0", C.c_double * 3),
                ("observer", C.c_double * 3), ("nb1", C.c_int32), ("nb2", C.c_int32),
                ("phi1_lo", C.c_double), ("phi1_hi", C.c_double),
                ("phi2_lo", C.c_double), ("phi2_hi", C.c_double)]


def make_params(G, eps, dt, checkpoint_every=0, ext_flags=0, nfw_M=0.0,
                nfw_rs=1.0, mn_M=0.0, mn_a=0.0, mn_b=0.0, center=(0, 0, 0),
                center_vel=(0, 0, 0), center_mode=NBODY_CENTER_FIXED,
                tape_mode=NBODY_TAPE_KEEP_LAST, bulge_M=0.0, bulge_alpha=1.8,
                bulge_rc=1.9) -> nbody_params:
    p = nbody_params()
    p.G, p.eps, p.dt = G, eps, dt
    p.checkpoint_every = int(checkpoint_every)
    p.ext_flags, p.center_mode, p.tape_mode, p.reserved = ext_flags, center_mode, tape_mode, 0
    p.nfw_M, p.nfw_rs, p.mn_M, p.mn_a, p.mn_b = nfw_M, nfw_rs, mn_M, mn_a, mn_b
    p.center[:] = [float(c) for c in center]
    p.center_vel[:] = [float(c) for c in center_vel]
    p.bulge_M, p.bulge_alpha, p.bulge_rc = bulge_M, bulge_alpha, bulge_rc
    return p


class NBodyError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, nbody_strerror(code), code))


_lib = None


def lib():
    """Load libnbody.so; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libnbody.so is not built (%s); run "
                               "paper_2511_22468_gb300.build.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        P = C.POINTER(nbody_params)
        vp, i64, dp = C.c_void_p, C.c_int64, C.POINTER(C.c_double)
        L.nbody_create.argtypes = [C.POINTER(vp), i64, P, vp]
        L.nbody_destroy.argtypes = [vp]
        L.nbody_destroy.restype = None
        L.nbody_set_params.argtypes = [vp, P]
        L.nbody_set_state.argtypes = [vp, vp, vp, vp]
        L.nbody_get_state.argtypes = [vp, vp, vp]
        L.nbody_step.argtypes = [vp, i64]
        L.nbody_integrate.argtypes = [vp, i64, vp, vp]
        L.nbody_vjp.argtypes = [vp, vp, vp, vp, vp, vp, dp]
        L.nbody_energy.argtypes = [vp, dp]
        L.nbody_momentum.argtypes = [vp, dp]
        L.nbody_get_status.argtypes = [vp]
        L.nbody_strerror.argtypes = [C.c_int]
        L.nbody_strerror.restype = C.c_char_p
        L.nbody_launch_count.argtypes = []
        L.nbody_launch_count.restype = i64
        L.nbody_pair_accel.argtypes = [i64, vp, vp, C.c_double, C.c_double,
                                       dp, vp, vp]
        L.nbody_pair_accel_noalloc.argtypes = [i64, vp, vp, C.c_double,
                                               C.c_double, dp, vp, vp]
        SC = C.POINTER(nbody_stream_cfg)
        L.nbody_stream_create.argtypes = [C.POINTER(vp), SC, vp, vp, vp]
        L.nbody_stream_set_target.argtypes = [vp, vp]
        L.nbody_stream_set_target_cloud.argtypes = [vp, i64, vp, vp, dp, C.c_int, dp]
        L.nbody_stream_initial_states.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.nbody_stream_autotune.argtypes = [vp, dp, C.c_int]
        L.nbody_stream_get_pair_shape.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
        L.nbody_stream_forward.argtypes = [vp, dp, dp, vp]
        L.nbody_stream_grad.argtypes = [vp, dp]
        L.nbody_stream_initial_state.argtypes = [vp, dp, vp, vp, vp, dp]
        L.nbody_stream_head.argtypes = [vp, vp, vp, dp]
        L.nbody_stream_destroy.argtypes = [vp]
        L.nbody_stream_destroy.restype = None
        L.nbody_create_batch.argtypes = [C.POINTER(vp), C.c_int, C.POINTER(i64), P, vp]
        L.nbody_vjp_batch.argtypes = [vp, vp, vp, vp, vp, vp]
        L.nbody_stream_batch_create.argtypes = [C.POINTER(vp), SC, i64, vp, vp, i64, vp, vp,
                                                dp, C.c_int, dp, vp]
        L.nbody_stream_batch_loss_grad.argtypes = [vp, vp, vp, vp]
        L.nbody_stream_batch_grad_parts.argtypes = [vp, vp]
        L.nbody_stream_batch_destroy.argtypes = [vp]
        L.nbody_stream_batch_destroy.restype = None
        L.nbody_autotune.argtypes = [vp, i64, C.POINTER(C.c_int), dp]
        L.nbody_set_tuning.argtypes = [vp, C.c_int]
        L.nbody_get_tuning.argtypes = [vp]
        fp = C.POINTER(C.c_float)
        L.nbody_mlp_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.c_int, vp]
        L.nbody_mlp_num_params.argtypes = [vp]
        L.nbody_mlp_num_params.restype = i64
        L.nbody_mlp_set_params.argtypes = [vp, vp]
        L.nbody_mlp_get_params.argtypes = [vp, vp]
        L.nbody_mlp_forward.argtypes = [vp, vp, C.c_int, vp]
        L.nbody_mlp_loss_grad.argtypes = [vp, vp, vp, C.c_int, fp, vp, vp]
        L.nbody_mlp_adam_step.argtypes = [vp, C.c_float, C.c_float, C.c_float, C.c_float]
        L.nbody_mlp_invert.argtypes = [vp, vp, C.c_int, vp, C.c_int, C.c_float,
                                        C.c_float, C.c_float, vp]
        L.nbody_mlp_get_status.argtypes = [vp]
        L.nbody_mlp_destroy.argtypes = [vp]
        L.nbody_mlp_destroy.restype = None
        L.nbody_set_pair_shape.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
        L.nbody_get_pair_shape.argtypes = [vp, C.c_int, C.POINTER(C.c_int)]
        L.nbody_set_pair_finish.argtypes = [vp, C.c_int, C.c_int]
        L.nbody_set_pair_tile.argtypes = [vp, C.c_int, C.c_int]
        L.nbody_get_pair_tile.argtypes = [vp, C.c_int]
        L.nbody_peaks.argtypes = [dp, vp]
        L.nbody_autotune_pair.argtypes = [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.nbody_set_timing.argtypes = [vp, C.c_int]
        L.nbody_kernel_times.argtypes = [vp, dp, C.POINTER(i64)]
        L.nbody_potential_grad.argtypes = [vp, dp]
        L.nbody_ext_accel.argtypes = [P, i64, vp, vp, vp]
        OC = C.POINTER(nbody_orbitfit_cfg)
        L.nbody_orbitfit_create.argtypes = [C.POINTER(vp), OC, i64, dp, vp]
        L.nbody_orbitfit_eval.argtypes = [vp, i64, dp, dp, dp, dp]
        L.nbody_orbitfit_lm.argtypes = [vp, i64, dp, C.c_int, dp, dp, dp, dp,
                                        C.POINTER(C.c_int)]
        L.nbody_orbitfit_fisher.argtypes = [vp, dp, dp, dp]
        L.nbody_orbitfit_arc.argtypes = [vp, dp, i64, dp, C.POINTER(i64)]
        L.nbody_orbitfit_destroy.argtypes = [vp]
        L.nbody_orbitfit_destroy.restype = None
        L.nbody_mmd_create.argtypes = [C.POINTER(vp), i64, i64, i64, vp, vp, dp, C.c_int,
                                       dp, vp]
        L.nbody_mmd_eval.argtypes = [vp, vp, vp, dp, vp, vp]
        L.nbody_mmd_eval_batch.argtypes = [vp, i64, vp, vp, vp]
        L.nbody_mmd_eval_cross.argtypes = [vp, i64, vp, vp, i64, i64, vp, vp, vp]
        L.nbody_mmd_target_stats.argtypes = [vp, dp, dp]
        L.nbody_mmd_destroy.argtypes = [vp]
        L.nbody_mmd_destroy.restype = None
        _lib = L
    return _lib


def _ptr(a, shape=None):
    """Raw address of a float64 contiguous torch tensor or numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 tensor")
        if shape is not None and tuple(a.shape) != tuple(shape):
            raise ValueError("expected shape %s, got %s" % (shape, tuple(a.shape)))
        return C.c_void_p(a.data_ptr())
    import numpy as np
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous float64 array")
    if shape is not None and tuple(a.shape) != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (shape, tuple(a.shape)))
    return C.c_void_p(a.ctypes.data)


def _fptr(a, shape=None):
    """Raw address of a float32 contiguous torch tensor or numpy array."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float32 or not a.is_contiguous():
            raise TypeError("expected a contiguous float32 tensor")
        if shape is not None and tuple(a.shape) != tuple(shape):
            raise ValueError("expected shape %s, got %s" % (shape, tuple(a.shape)))
        return C.c_void_p(a.data_ptr())
    import numpy as np
    if a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"]:
        raise TypeError("expected a C-contiguous float32 array")
    return C.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _check(rc, what):
    if rc != NBODY_OK:
        raise NBodyError(rc, what)


def nbody_strerror(code: int) -> str:
    return lib().nbody_strerror(code).decode()


def nbody_launch_count() -> int:
    return lib().nbody_launch_count()


def nbody_create(n: int, params: nbody_params, stream=None):
    h = C.c_void_p()
    _check(lib().nbody_create(C.byref(h), n, C.byref(params), _stream(stream)),
           "nbody_create")
    return h


def nbody_destroy(h):
    lib().nbody_destroy(h)


def nbody_set_params(h, params: nbody_params):
    _check(lib().nbody_set_params(h, C.byref(params)), "nbody_set_params")


def nbody_set_state(h, x, v, m):
    n = m.shape[0]
    _check(lib().nbody_set_state(h, _ptr(x, (3, n)), _ptr(v, (3, n)), _ptr(m, (n,))),
           "nbody_set_state")


def nbody_get_state(h, x=None, v=None):
    _check(lib().nbody_get_state(h, _ptr(x), _ptr(v)), "nbody_get_state")


def nbody_step(h, k: int):
    _check(lib().nbody_step(h, k), "nbody_step")


def nbody_integrate(h, n_steps: int, x_out=None, v_out=None):
    _check(lib().nbody_integrate(h, n_steps, _ptr(x_out), _ptr(v_out)),
           "nbody_integrate")


def nbody_vjp(h, xbar, vbar, x0bar=None, v0bar=None, mbar=None):
    """Returns theta_bar = (dL/d dt, sum_j m_j dL/dm_j, dL/dM_NFW, dL/dM_MN);
    fills x0bar, v0bar (3, n) and mbar (n,) when given."""
    tb = (C.c_double * 4)()
    _check(lib().nbody_vjp(h, _ptr(xbar), _ptr(vbar), _ptr(x0bar), _ptr(v0bar),
                           _ptr(mbar), tb), "nbody_vjp")
    return list(tb)


def nbody_potential_grad(h):
    """(dL/dM_NFW, dL/dr_s, dL/dM_MN, dL/da_MN, dL/db_MN, dL/dM_bulge) of the
    last vjp."""
    out = (C.c_double * 6)()
    _check(lib().nbody_potential_grad(h, out), "nbody_potential_grad")
    return list(out)


def nbody_mmd_create(n, max_sets, tx, tv, sigmas, scale=None, stream=None):
    """MMD evaluator for clouds of n points against the target (tx, tv:
    (3, m) each)."""
    m = tx.shape[1]
    h = C.c_void_p()
    sg = (C.c_double * len(sigmas))(*[float(s) for s in sigmas])
    sc = None if scale is None else (C.c_double * 6)(*[float(s) for s in scale])
    _check(lib().nbody_mmd_create(C.byref(h), n, max_sets, m, _ptr(tx, (3, m)),
                                  _ptr(tv, (3, m)), sc, len(sigmas), sg, _stream(stream)),
           "nbody_mmd_create")
    return h


def nbody_mmd_eval(h, x, v, xbar=None, vbar=None):
    loss = C.c_double()
    _check(lib().nbody_mmd_eval(h, _ptr(x), _ptr(v), C.byref(loss), _ptr(xbar), _ptr(vbar)),
           "nbody_mmd_eval")
    return loss.value


def nbody_mmd_eval_batch(h, sets, x, v, losses):
    _check(lib().nbody_mmd_eval_batch(h, sets, _ptr(x), _ptr(v), _ptr(losses)),
           "nbody_mmd_eval_batch")


def nbody_mmd_eval_cross(h, sets, x, v, targets, m2, ty, tv, losses):
    """MMD^2 of `sets` clouds against each of `targets` clouds of m2 points;
    losses[t * sets + b]."""
    _check(lib().nbody_mmd_eval_cross(h, sets, _ptr(x), _ptr(v), targets, m2, _ptr(ty),
                                      _ptr(tv), _ptr(losses)), "nbody_mmd_eval_cross")


def nbody_mmd_target_stats(h):
    mu = (C.c_double * 6)()
    sc = (C.c_double * 6)()
    _check(lib().nbody_mmd_target_stats(h, mu, sc), "nbody_mmd_target_stats")
    return list(mu), list(sc)


def nbody_mmd_destroy(h):
    lib().nbody_mmd_destroy(h)


def nbody_energy(h):
    """(K, W_pair, W_ext, |P|)."""
    out = (C.c_double * 4)()
    _check(lib().nbody_energy(h, out), "nbody_energy")
    return list(out)


def nbody_momentum(h):
    out = (C.c_double * 3)()
    _check(lib().nbody_momentum(h, out), "nbody_momentum")
    return list(out)


def nbody_get_status(h) -> int:
    return lib().nbody_get_status(h)


def nbody_pair_accel(x, m, G, eps, center, acc, stream=None):
    """a_i of the softened pair sum for device tensors x (3, n), m (n,)
    into acc (3, n)."""
    n = m.shape[0]
    cen = (C.c_double * 3)(*[float(c) for c in center])
    _check(lib().nbody_pair_accel(n, _ptr(x, (3, n)), _ptr(m, (n,)), G, eps,
                                  cen, _ptr(acc, (3, n)), _stream(stream)),
           "nbody_pair_accel")


def nbody_ext_accel(params, x, acc, stream=None):
    """External acceleration at the points x (3, n) into acc (3, n)."""
    n = x.shape[1]
    _check(lib().nbody_ext_accel(C.byref(params), n, _ptr(x, (3, n)), _ptr(acc, (3, n)),
                                 _stream(stream)), "nbody_ext_accel")


def nbody_pair_accel_noalloc(x, m, G, eps, center, acc, stream=None):
    """nbody_pair_accel without device allocation, for callers that cannot
    allocate when they need forces (fixed up-front memory budget, or a loop
    that must avoid the allocator); scratch lives in a fixed 4 MiB device
    array of the library, n <= NBODY_NOALLOC_MAX_N.  Asynchronous on the
    stream; calls overlapping on the GPU race on the shared array."""
    n = m.shape[0]
    cen = (C.c_double * 3)(*[float(c) for c in center])
    _check(lib().nbody_pair_accel_noalloc(n, _ptr(x, (3, n)), _ptr(m, (n,)), G, eps,
                                          cen, _ptr(acc, (3, n)), _stream(stream)),
           "nbody_pair_accel_noalloc")


def nbody_set_pair_shape(h, vjp, variant, threads, per_thread, chunks=0):
    _check(lib().nbody_set_pair_shape(h, int(vjp), variant, threads, per_thread, chunks),
           "nbody_set_pair_shape")


def nbody_set_pair_finish(h, vjp, mode):
    """Chunk sums added in the pair kernel (1), by the consumer (0) or by
    chunk count (-1); results are bitwise the same."""
    _check(lib().nbody_set_pair_finish(h, int(vjp), int(mode)), "nbody_set_pair_finish")


def nbody_set_pair_tile(h, vjp, tile_pairs):
    """j-pairs per shared-memory tile of the tile variant (default or 128)."""
    _check(lib().nbody_set_pair_tile(h, int(vjp), int(tile_pairs)), "nbody_set_pair_tile")


def nbody_get_pair_tile(h, vjp):
    rc = lib().nbody_get_pair_tile(h, int(vjp))
    _check(rc if rc < 0 else 0, "nbody_get_pair_tile")
    return rc


def nbody_get_pair_shape(h, vjp):
    """(variant, threads, per_thread, chunks)."""
    out = (C.c_int * 4)()
    _check(lib().nbody_get_pair_shape(h, int(vjp), out), "nbody_get_pair_shape")
    return tuple(out)


def nbody_autotune_pair(h, probe_launches=3):
    """Tune the single-system pair kernels; returns (forward shape, VJP shape)."""
    f = (C.c_int * 4)()
    v = (C.c_int * 4)()
    _check(lib().nbody_autotune_pair(h, probe_launches, f, v), "nbody_autotune_pair")
    return tuple(f), tuple(v)


def nbody_peaks(stream=None):
    """dict of measured unit throughputs of the current device."""
    out = (C.c_double * 6)()
    _check(lib().nbody_peaks(out, _stream(stream)), "nbody_peaks")
    return {"fp32_fma_tflops": out[0], "fp32x2_fma_tflops": out[1],
            "fp64_fma_tflops": out[2], "rsqrt_gops": out[3], "sms": int(out[4]),
            "ex2_gops": out[5]}


def nbody_set_timing(h, enable: bool):
    _check(lib().nbody_set_timing(h, int(bool(enable))), "nbody_set_timing")


def nbody_kernel_times(h):
    """{class: (ms, launches)} summed since the previous call."""
    ms = (C.c_double * len(NBODY_KCLASS))()
    cnt = (C.c_int64 * len(NBODY_KCLASS))()
    _check(lib().nbody_kernel_times(h, ms, cnt), "nbody_kernel_times")
    return {k: (ms[i], cnt[i]) for i, k in enumerate(NBODY_KCLASS)}


def nbody_create_batch(offsets, params_list, stream=None):
    """Batch context for len(params_list) simulations; offsets has one more
    entry (particle ranges of the concatenated state)."""
    ns = len(params_list)
    offs = (C.c_int64 * (ns + 1))(*[int(o) for o in offsets])
    arr = (nbody_params * ns)(*params_list)
    h = C.c_void_p()
    _check(lib().nbody_create_batch(C.byref(h), ns, offs, arr, _stream(stream)),
           "nbody_create_batch")
    return h


def nbody_vjp_batch(h, n_sims, xbar, vbar, x0bar=None, v0bar=None):
    """Adjoint of a batch's last recorded run: fills x0bar, v0bar (3, ntot)
    when given and returns theta_bar (n_sims, 8) = per simulation (dL/d dt,
    sum_j m_j dL/dm_j, dL/dM_NFW, dL/dM_MN, dL/dr_s, dL/da_MN, dL/db_MN,
    dL/dM_bulge)."""
    import numpy as np
    tb = np.zeros((n_sims, 8))
    _check(lib().nbody_vjp_batch(h, _ptr(xbar), _ptr(vbar), _ptr(x0bar), _ptr(v0bar),
                                 _ptr(tb)), "nbody_vjp_batch")
    return tb


def nbody_stream_batch_create(cfg, count, xhat, vhat, m, tx, tv, scale, sigmas, stream=None):
    """Pipeline of `count` parameter vectors, member b against target b
    (tx, tv: (3, count m))."""
    h = C.c_void_p()
    n = cfg.n
    sc = (C.c_double * 6)(*[float(v) for v in scale])
    sg = (C.c_double * len(sigmas))(*[float(v) for v in sigmas])
    _check(lib().nbody_stream_batch_create(C.byref(h), C.byref(cfg), count, _ptr(xhat, (3, n)),
                                           _ptr(vhat, (3, n)), m, _ptr(tx, (3, count * m)),
                                           _ptr(tv, (3, count * m)), sc, len(sigmas), sg,
                                           _stream(stream)), "nbody_stream_batch_create")
    return h


def nbody_stream_batch_grad_parts(h, count):
    """(count, 2, 4): the two parts of every component of the last gradient
    (n-body run / velocity scaling, then orbit / masses)."""
    import numpy as np
    out = np.zeros((count, 8))
    _check(lib().nbody_stream_batch_grad_parts(h, _ptr(out)), "nbody_stream_batch_grad_parts")
    return out.reshape(count, 2, 4)


def nbody_stream_batch_loss_grad(h, thetas, want_grad=True):
    """(losses (count,), dL/dtheta (count, 4) or None) at thetas (count, 4)."""
    import numpy as np
    th = np.ascontiguousarray(np.asarray(thetas, np.float64))
    L = np.empty(th.shape[0])
    g = np.empty_like(th) if want_grad else None
    _check(lib().nbody_stream_batch_loss_grad(h, _ptr(th), _ptr(L), _ptr(g)),
           "nbody_stream_batch_loss_grad")
    return L, g


def nbody_stream_batch_destroy(h):
    lib().nbody_stream_batch_destroy(h)


def nbody_set_params_batch(h, params_list):
    arr = (nbody_params * len(params_list))(*params_list)
    _check(lib().nbody_set_params(h, arr), "nbody_set_params")


def nbody_autotune(h, probe_steps=3):
    """(best candidate, [ms per launch of each candidate])."""
    best = C.c_int()
    ms = (C.c_double * NBODY_NTUNE)()
    _check(lib().nbody_autotune(h, probe_steps, C.byref(best), ms), "nbody_autotune")
    return best.value, list(ms)


def nbody_set_tuning(h, choice):
    _check(lib().nbody_set_tuning(h, int(choice)), "nbody_set_tuning")


def nbody_get_tuning(h):
    rc = lib().nbody_get_tuning(h)
    if rc < 0:
        raise NBodyError(rc, "nbody_get_tuning")
    return rc


def nbody_mlp_create(n_in, n_hidden, n_out, max_batch, stream=None):
    h = C.c_void_p()
    _check(lib().nbody_mlp_create(C.byref(h), n_in, n_hidden, n_out, max_batch,
                                  _stream(stream)), "nbody_mlp_create")
    return h


def nbody_mlp_num_params(h):
    return lib().nbody_mlp_num_params(h)


def nbody_mlp_set_params(h, params):
    _check(lib().nbody_mlp_set_params(h, _fptr(params)), "nbody_mlp_set_params")


def nbody_mlp_get_params(h, params):
    _check(lib().nbody_mlp_get_params(h, _fptr(params)), "nbody_mlp_get_params")


def nbody_mlp_forward(h, u, y):
    _check(lib().nbody_mlp_forward(h, _fptr(u), u.shape[0], _fptr(y)), "nbody_mlp_forward")


def nbody_mlp_loss_grad(h, u, t, grads=None, du=None, want_loss=True):
    loss = C.c_float()
    _check(lib().nbody_mlp_loss_grad(h, _fptr(u), _fptr(t), u.shape[0],
                                     C.byref(loss) if want_loss else None,
                                     _fptr(grads), _fptr(du)), "nbody_mlp_loss_grad")
    return loss.value if want_loss else None


def nbody_mlp_adam_step(h, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(lib().nbody_mlp_adam_step(h, lr, beta1, beta2, eps), "nbody_mlp_adam_step")


def nbody_mlp_invert(h, target, u, iters, lr, lo=-1.5, hi=1.5, loss=None):
    """Adam on the inputs u (starts, n_in) toward target (n_out,); in place."""
    _check(lib().nbody_mlp_invert(h, _fptr(target), u.shape[0], _fptr(u), iters, lr, lo,
                                  hi, _fptr(loss)), "nbody_mlp_invert")


def nbody_mlp_get_status(h):
    """NBODY_OK, or NBODY_ETIMEOUT after an expired tensor-core wait."""
    return lib().nbody_mlp_get_status(h)


def nbody_mlp_destroy(h):
    lib().nbody_mlp_destroy(h)


def nbody_stream_create(cfg: nbody_stream_cfg, xhat, vhat, stream=None):
    h = C.c_void_p()
    n = cfg.n
    _check(lib().nbody_stream_create(C.byref(h), C.byref(cfg), _ptr(xhat, (3, n)),
                                     _ptr(vhat, (3, n)), _stream(stream)),
           "nbody_stream_create")
    return h


def nbody_stream_set_target(h, target):
    _check(lib().nbody_stream_set_target(h, _ptr(target)), "nbody_stream_set_target")


def nbody_stream_set_target_cloud(h, tx, tv, sigmas, scale=None):
    """Point-cloud (MMD) loss against the cloud tx, tv ((3, m) each)."""
    m = tx.shape[1]
    sg = (C.c_double * len(sigmas))(*[float(s) for s in sigmas])
    sc = None if scale is None else (C.c_double * 6)(*[float(s) for s in scale])
    _check(lib().nbody_stream_set_target_cloud(h, m, _ptr(tx, (3, m)), _ptr(tv, (3, m)), sc,
                                               len(sigmas), sg),
           "nbody_stream_set_target_cloud")


def nbody_stream_forward(h, theta, density=None):
    """Loss at theta = (t_end, M_Plummer, M_NFW, M_MN); fills density if given."""
    th = (C.c_double * 4)(*[float(t) for t in theta])
    loss = C.c_double()
    _check(lib().nbody_stream_forward(h, th, C.byref(loss), _ptr(density)),
           "nbody_stream_forward")
    return loss.value


def nbody_stream_grad(h):
    tb = (C.c_double * 4)()
    _check(lib().nbody_stream_grad(h, tb), "nbody_stream_grad")
    return list(tb)


def nbody_stream_initial_state(h, theta, x0, v0, m):
    """Fills x0, v0 (3, n) and m (n,) on the device; returns the recovered
    centre of mass (X, V) as 6 floats."""
    th = (C.c_double * 4)(*[float(t) for t in theta])
    com = (C.c_double * 6)()
    _check(lib().nbody_stream_initial_state(h, th, _ptr(x0), _ptr(v0), _ptr(m), com),
           "nbody_stream_initial_state")
    return list(com)


def nbody_stream_initial_states(h, thetas, x0, v0, m, com=None):
    """Initial states of count = len(thetas) parameter vectors: x0, v0
    (3, count n) and m (count n,) on the device; com (count, 6) if given."""
    import numpy as np
    th = np.ascontiguousarray(np.asarray(thetas, np.float64).reshape(-1, 4))
    _check(lib().nbody_stream_initial_states(h, th.shape[0], _ptr(th), _ptr(x0), _ptr(v0),
                                             _ptr(m), _ptr(com)),
           "nbody_stream_initial_states")


def nbody_stream_autotune(h, theta, probe_launches=3):
    th = (C.c_double * 4)(*[float(t) for t in theta])
    _check(lib().nbody_stream_autotune(h, th, int(probe_launches)), "nbody_stream_autotune")


def nbody_stream_get_pair_shape(h, vjp):
    """(variant, threads, per_thread, chunks) of the pipeline's pair-force
    (vjp = 0) or pair-VJP (vjp = 1) kernel."""
    out = (C.c_int * 4)()
    _check(lib().nbody_stream_get_pair_shape(h, int(vjp), out), "nbody_stream_get_pair_shape")
    return tuple(out)


def nbody_stream_head(h, x, density, want_loss=False):
    loss = C.c_double()
    _check(lib().nbody_stream_head(h, _ptr(x), _ptr(density),
                                   C.byref(loss) if want_loss else None),
           "nbody_stream_head")
    return loss.value if want_loss else None


def nbody_stream_destroy(h):
    lib().nbody_stream_destroy(h)


class Simulation:
    """Owning wrapper of one context (create / destroy)."""

    def __init__(self, n, params, stream=None):
        self.n = n
        self.params = params
        self.h = nbody_create(n, params, stream)

    def close(self):
        if self.h is not None and self.h.value:
            nbody_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        self.params = params
        nbody_set_params(self.h, params)

    def set_state(self, x, v, m):
        nbody_set_state(self.h, x, v, m)

    def get_state(self, x=None, v=None):
        nbody_get_state(self.h, x, v)

    def step(self, k):
        nbody_step(self.h, k)

    def integrate(self, n_steps, x_out=None, v_out=None):
        nbody_integrate(self.h, n_steps, x_out, v_out)

    def vjp(self, xbar, vbar, x0bar=None, v0bar=None, mbar=None):
        return nbody_vjp(self.h, xbar, vbar, x0bar, v0bar, mbar)

    def potential_grad(self):
        return nbody_potential_grad(self.h)

    def energy(self):
        return nbody_energy(self.h)

    def momentum(self):
        return nbody_momentum(self.h)

    def status(self):
        return nbody_get_status(self.h)


_RUN_FN = None


def _run_fn():
    global _RUN_FN
    if _RUN_FN is None:
        import torch

        class _Run(torch.autograd.Function):
            @staticmethod
            def forward(ctx, x0, v0, m, theta, sim, n_steps):
                if theta is not None:
                    t = [float(a) for a in theta.detach().cpu().tolist()]
                    p = sim.params
                    p.dt, p.nfw_M, p.nfw_rs, p.mn_M, p.mn_a, p.mn_b = t
                    sim.set_params(p)
                sim.set_state(x0.detach().contiguous(), v0.detach().contiguous(),
                              m.detach().contiguous())
                xT = torch.empty_like(x0)
                vT = torch.empty_like(v0)
                sim.integrate(n_steps, xT, vT)
                ctx.sim = sim
                ctx.theta_like = theta
                return xT, vT

            @staticmethod
            def backward(ctx, xbar, vbar):
                sim = ctx.sim
                like = xbar if xbar is not None else vbar
                xbar = torch.zeros_like(like) if xbar is None else xbar.contiguous()
                vbar = torch.zeros_like(like) if vbar is None else vbar.contiguous()
                want = ctx.needs_input_grad
                x0b = torch.empty_like(xbar) if want[0] else None
                v0b = torch.empty_like(xbar) if want[1] else None
                mb = (torch.empty(xbar.shape[1], dtype=xbar.dtype, device=xbar.device)
                      if want[2] else None)
                tb = sim.vjp(xbar, vbar, x0b, v0b, mb)
                thb = None
                if want[3]:
                    th = ctx.theta_like
                    thb = torch.tensor([tb[0]] + sim.potential_grad()[:5], dtype=th.dtype,
                                       device=th.device)
                return x0b, v0b, mb, thb, None, None

        _RUN_FN = _Run
    return _RUN_FN


def simulate(sim: Simulation, x0, v0, m, n_steps: int, theta=None):
    """Differentiable run of one context: (x_T, v_T), each (3, n) FP64 on the
    device of x0, with a torch autograd backward through nbody_vjp that gives
    dL/dx0, dL/dv0, dL/dm and, when theta = (dt, M_NFW, r_s, M_MN, a_MN,
    b_MN) is passed as a tensor (its values then replace the context's),
    dL/dtheta.  The tape
    lives in the context: run the backward before the context's next
    integration."""
    return _run_fn().apply(x0, v0, m, theta, sim, int(n_steps))


# ---- orbit fitting (host numpy arrays in and out) ----
def _dp(a):
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def nbody_orbitfit_create(cfg: nbody_orbitfit_cfg, obs, stream=None):
    import numpy as np
    obs, po = _dp(np.asarray(obs, float).reshape(-1, 5))
    h = C.c_void_p()
    _check(lib().nbody_orbitfit_create(C.byref(h), C.byref(cfg), obs.shape[0], po,
                                       _stream(stream)), "nbody_orbitfit_create")
    return h


def nbody_orbitfit_eval(h, thetas, want_grad=True, want_gn=True):
    """(chi2 (k,), grad (k, 5) or None, gn (k, 5, 5) or None)."""
    import numpy as np
    th, pt = _dp(np.asarray(thetas, float).reshape(-1, 5))
    k = th.shape[0]
    chi2, pc = _dp(np.zeros(k))
    g, pg = _dp(np.zeros((k, 5))) if want_grad else (None, None)
    a, pa = _dp(np.zeros((k, 5, 5))) if want_gn else (None, None)
    _check(lib().nbody_orbitfit_eval(h, k, pt, pc, pg, pa), "nbody_orbitfit_eval")
    return chi2, g, a


def nbody_orbitfit_lm(h, theta0, max_iter=100, lo=None, hi=None):
    """(theta (k, 5), chi2 (k,), iterations (k,)); lo, hi: optional box."""
    import numpy as np
    th, pt = _dp(np.asarray(theta0, float).reshape(-1, 5))
    k = th.shape[0]
    out, po = _dp(np.zeros((k, 5)))
    chi2, pc = _dp(np.zeros(k))
    its = (C.c_int * k)()
    lo_a, plo = _dp(np.asarray(lo, float).reshape(5)) if lo is not None else (None, None)
    hi_a, phi = _dp(np.asarray(hi, float).reshape(5)) if hi is not None else (None, None)
    _check(lib().nbody_orbitfit_lm(h, k, pt, int(max_iter), plo, phi, po, pc, its),
           "nbody_orbitfit_lm")
    return out, chi2, np.array(its[:], dtype=int)


def nbody_orbitfit_fisher(h, theta):
    """(F, F_gn), 5 x 5 each, in ln theta."""
    import numpy as np
    th, pt = _dp(np.asarray(theta, float).reshape(5))
    F, pf = _dp(np.zeros((5, 5)))
    Fg, pg = _dp(np.zeros((5, 5)))
    _check(lib().nbody_orbitfit_fisher(h, pt, pf, pg), "nbody_orbitfit_fisher")
    return F, Fg


def nbody_orbitfit_arc(h, theta, max_pts=20000):
    import numpy as np
    th, pt = _dp(np.asarray(theta, float).reshape(5))
    arc, pa = _dp(np.zeros((max_pts, 5)))
    n = C.c_int64()
    _check(lib().nbody_orbitfit_arc(h, pt, max_pts, pa, C.byref(n)), "nbody_orbitfit_arc")
    return arc[:n.value].copy()


def nbody_orbitfit_destroy(h):
    lib().nbody_orbitfit_destroy(h)

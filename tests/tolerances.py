"""Error measures shared by the GPU parity tests.

Every per-particle quantity (acceleration, gradient with respect to a
particle's position, velocity or mass) is compared particle by particle,
relative to its own size with a floor of 1e-3 of the array's rms size, so
that a particle whose value is near zero is not held to an unattainable
relative bound while every other particle is held to the full one.
"""
import numpy as np


def per_particle_err(got, ref, floor=1e-3):
    """max_k |got_k - ref_k| / (|ref_k| + floor * rms_k |ref_k|): rows of
    (n, d) arrays by their vector norm, entries of (n,) arrays by absolute
    value."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if ref.ndim == 2:
        size = np.linalg.norm(ref, axis=1)
        diff = np.linalg.norm(got - ref, axis=1)
    else:
        size = np.abs(ref)
        diff = np.abs(got - ref)
    scale = size + floor * np.sqrt(np.mean(size * size))
    return float(np.max(diff / scale))


U32 = 2.0 ** -24  # FP32 unit roundoff


def mass_grad_abs_terms(x, G, eps, lam, rows=None, chunk=256):
    """A_k = G sum_i |lam_i . (x_k - x_i)| / s_ik^3 (FP64): the sum of the
    absolute values of the terms whose signed sum is the per-particle mass
    gradient sum_i lam_i . d a_i / d m_k.  It is the scale of the FP32
    rounding error of that sum (an error-bound scale for the tests, not an
    expected value)."""
    x = np.asarray(x, np.float64)
    lam = np.asarray(lam, np.float64)
    sel = np.arange(x.shape[0]) if rows is None else np.asarray(rows)
    out = np.empty(sel.shape[0])
    for a in range(0, sel.shape[0], chunk):
        k = sel[a:a + chunk]
        d = x[k][:, None, :] - x[None, :, :]
        s3 = (np.sum(d * d, axis=2) + eps * eps) ** 1.5
        out[a:a + chunk] = G * np.sum(np.abs(np.einsum("kic,ic->ki", d, lam)) / s3, axis=1)
    return out


def per_particle_err_fp32_sum(got, ref, abs_terms, rel=1e-4, floor=1e-3, c=8.0):
    """max_k |got_k - ref_k| / (rel (|ref_k| + floor rms|ref|) + c u A_k) for
    per-particle sums of terms of either sign computed with FP32 terms
    (u = 2^-24, A_k the sum of the terms' absolute values): the relative
    bound where the sum is well conditioned, the FP32 summation error bound
    c u A_k where cancellation leaves the sum far below its terms.  Pass
    when <= 1."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    size = np.abs(ref)
    scale = rel * (size + floor * np.sqrt(np.mean(size * size))) + c * U32 * np.asarray(abs_terms)
    return float(np.max(np.abs(got - ref) / scale))

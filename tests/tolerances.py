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

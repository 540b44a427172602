"""Host logic of the refinement stage (no GPU): the batched Adam descent
against the one-problem descent on the same problems, and the seeded
realisations of an observation."""
import numpy as np
import pytest

pytest.importorskip("torch")

from paper_2511_22468_gb300.inputs import perturbed_clouds  # noqa: E402
from paper_2511_22468_gb300.surrogate import descend, descend_batch  # noqa: E402


class Bowl:
    """L(theta) = sum_k w_k (theta_k / c_k - 1 - s_k)^2 + ripple, one bowl per
    problem; the ripple makes some Adam steps overshoot, so the undo branch
    runs too."""

    def __init__(self, centre, shift, weight):
        self.c, self.s, self.w = (np.asarray(a, float) for a in (centre, shift, weight))

    def _one(self, th, s, w):
        q = th / self.c - 1.0 - s
        L = np.sum(w * q * q) + 0.05 * np.sum(np.sin(40.0 * q) ** 2)
        g = (2.0 * w * q + 0.05 * 80.0 * np.sin(40.0 * q) * np.cos(40.0 * q)) / self.c
        return L, g

    def loss_and_grad(self, theta):
        th = np.asarray(theta, float)
        if th.ndim == 1:
            return self._one(th, self.s[0], self.w[0])
        out = [self._one(t, s, w) for t, s, w in zip(th, self.s, self.w)]
        return np.array([o[0] for o in out]), np.array([o[1] for o in out])


def test_batched_descent_equals_one_problem_descent():
    rng = np.random.default_rng(3)
    centre = np.array([500.0, 2e4, 1e12, 7e10])
    shifts = rng.uniform(-0.2, 0.2, (6, 4))
    weights = rng.uniform(0.5, 3.0, (6, 4))
    starts = centre[None, :] * rng.uniform(0.8, 1.2, (6, 4))
    best, Lb, trace = descend_batch(Bowl(centre, shifts, weights), starts, centre, 0.3,
                                    lr=0.05, iters=12)
    undone = 0
    for b in range(6):
        one = Bowl(centre, shifts[b:b + 1], weights[b:b + 1])
        tr = descend(one, starts[b], centre, 0.3, lr=0.05, max_iters=12)
        undone += tr[-1]["lr"] < 0.05
        np.testing.assert_allclose(best[b], tr[-1]["theta"], rtol=1e-12)
        assert Lb[b] == pytest.approx(tr[-1]["loss"], rel=1e-12)
        np.testing.assert_allclose(trace[:, b], [r["loss"] for r in tr], rtol=1e-12)
    assert np.all(np.diff(trace, axis=0) <= 0.0)
    assert undone > 0   # some problems took the undo-and-halve branch


def test_perturbed_clouds_are_seeded_gaussian_redraws():
    rng = np.random.default_rng(0)
    x, v = rng.normal(size=(500, 3)), rng.normal(size=(500, 3)) * 1e-2
    rx, rv = perturbed_clouds(x, v, 0.1, np.array([1e-3, 2e-3, 3e-3]), 40, seed=9)
    rx2, rv2 = perturbed_clouds(x, v, 0.1, np.array([1e-3, 2e-3, 3e-3]), 40, seed=9)
    assert rx.shape == (40, 500, 3) and np.array_equal(rx, rx2) and np.array_equal(rv, rv2)
    ex, ev = rx - x[None], rv - v[None]
    assert abs(ex.std() - 0.1) < 0.002 and abs(ex.mean()) < 0.002
    np.testing.assert_allclose(ev.std(axis=(0, 1)), [1e-3, 2e-3, 3e-3], rtol=0.03)
    assert not np.array_equal(perturbed_clouds(x, v, 0.1, 1e-3, 1, seed=10)[0][0], rx[0])

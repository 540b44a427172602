"""Host logic of the grid stage (no GPU): pattern_search against a fake
batch whose loss is a known quadratic in the parameters."""
import numpy as np

from paper_2511_22468_gb300.surrogate import to_u
from paper_2511_22468_gb300.warmstart import pattern_search

CENTRE = np.array([3000.0, 2e4, 1e12, 6.8e10])
WIDTH = 0.3


class FakeBatch:
    """loss(thetas) = sum_k (w_k (theta_k / theta*_k - 1))^2 for every row."""

    def __init__(self, theta_star, w=(1.0, 0.5, 2.0, 0.2)):
        self.theta_star = np.asarray(theta_star, float)
        self.w = np.asarray(w, float)
        self.calls = []

    def loss(self, thetas):
        thetas = np.asarray(thetas, float)
        self.calls.append(thetas.copy())
        return np.sum((self.w * (thetas / self.theta_star - 1.0)) ** 2, axis=1)


def test_reaches_the_target_from_the_prior_centre():
    star = CENTRE * np.array([1.15, 0.85, 1.2, 0.8])
    fb = FakeBatch(star)
    tr = pattern_search(fb, CENTRE, WIDTH, star, 0.05, s0=0.37, max_calls=40)
    assert tr[-1]["err"] <= 0.05
    assert all(c.shape == (81, 4) for c in fb.calls)        # 3^4 points per call
    losses = [r["loss"] for r in tr]
    assert all(b <= a for a, b in zip(losses, losses[1:]))  # best-so-far never rises


def test_start_point_and_spacing_per_parameter():
    star = CENTRE * np.array([1.05, 0.97, 1.02, 0.9])
    fb = FakeBatch(star)
    u0 = np.array([0.2, -0.1, 0.05, -0.3])
    s0 = np.array([0.1, 0.2, 0.3, 0.4])
    pattern_search(fb, CENTRE, WIDTH, star, 0.0, s0=s0, max_calls=1, u_start=u0)
    U = to_u(fb.calls[0], CENTRE, WIDTH)
    np.testing.assert_allclose(U.mean(axis=0), u0, atol=1e-12)     # centred on u_start
    for k in range(4):                                             # offsets -s, 0, +s
        np.testing.assert_allclose(np.unique(np.round(U[:, k] - u0[k], 12)),
                                   [-s0[k], 0.0, s0[k]], atol=1e-12)


def test_spacing_halves_when_the_centre_is_best():
    fb = FakeBatch(CENTRE)          # the optimum is the start itself
    tr = pattern_search(fb, CENTRE, WIDTH, CENTRE, -1.0, s0=0.4, s_min=0.02, max_calls=30)
    sp = [r["spacing"][0] for r in tr]
    np.testing.assert_allclose(sp, [0.4 * 0.5 ** (i + 1) for i in range(len(sp))])
    assert sp[-1] < 0.02 <= sp[-2] and all(r["err"] == 0.0 for r in tr)

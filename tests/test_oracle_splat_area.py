"""Pins of the oracle's rendering-cost term (splat footprint relative to a
reference estimate): a hand-computed case, finite differences, and the
points whose reference area is degenerate."""
import numpy as np

from oracle.mlp import splat_area_loss


def test_hand_case():
    s = np.array([[2.0, 3.0, 0.1], [1.0, 1.0, 1.0]])
    r = np.array([[1.0, 2.0, 0.5], [0.5, 0.5, 0.5]])
    a, d = splat_area_loss(s, r, 0.5)
    # ratios 6 / 2 = 3 and 1 / 0.25 = 4; mean 3.5; times 0.5
    assert abs(a - 1.75) < 1e-15
    np.testing.assert_allclose(d, [[0.25 * 3.0 / 2.0, 0.25 * 2.0 / 2.0, 0.0],
                                   [0.25 * 1.0 / 0.25, 0.25 * 1.0 / 0.25, 0.0]], rtol=1e-15)


def test_finite_differences():
    rng = np.random.default_rng(3)
    s = rng.uniform(0.001, 0.02, (40, 3))
    r = rng.uniform(0.001, 0.02, (40, 3))
    a0, d = splat_area_loss(s, r, 0.3)
    h = 1e-7
    for i, k in [(0, 0), (5, 1), (17, 0), (39, 1), (3, 2)]:
        sp, sm = s.copy(), s.copy()
        sp[i, k] += h
        sm[i, k] -= h
        fd = (splat_area_loss(sp, r, 0.3)[0] - splat_area_loss(sm, r, 0.3)[0]) / (2 * h)
        assert abs(fd - d[i, k]) <= 1e-6 * max(1.0, abs(d[i, k])), (i, k, fd, d[i, k])


def test_degenerate_reference_adds_nothing():
    s = np.array([[1.0, 1.0, 1.0], [2.0, 2.0, 2.0], [3.0, 3.0, 3.0]])
    r = np.array([[1.0, 1.0, 1.0], [0.0, 1.0, 1.0], [np.inf, 1.0, 1.0]])
    a, d = splat_area_loss(s, r, 1.0)
    assert abs(a - 1.0 / 3.0) < 1e-15  # only the first point, over n = 3
    assert not d[1:].any()

"""Pins of the SSIM oracle (oracle/ssim.py) against what the definition
fixes independently of the oracle's own code."""
import numpy as np
import pytest

import oracle.ssim as os_


def test_window_is_scipy_gaussian():
    scipy_nd = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(0)
    img = rng.random((23, 31))
    # scipy's Gaussian filter with the same radius (truncate * sigma = 5)
    # and zero padding: the same normalised 11-tap kernel
    ref = scipy_nd.gaussian_filter(img, sigma=1.5, truncate=5 / 1.5, mode="constant", cval=0.0)
    np.testing.assert_allclose(os_.blur(img), ref, rtol=0, atol=1e-14)


def test_identical_images():
    rng = np.random.default_rng(1)
    x = rng.random((3, 17, 13))
    d, g = os_.loss_and_grad([x], [x.copy()])
    assert abs(d) < 1e-14
    assert np.abs(g[0]).max() < 1e-14


def test_constant_images_closed_form():
    a, b = 0.3, 0.7
    x = np.full((1, 40, 40), a)
    y = np.full((1, 40, 40), b)
    S = os_.ssim_terms(x[0], y[0])["S"]
    # away from the zero-padded border: no variance, the luminance term only
    interior = S[6:-6, 6:-6]
    np.testing.assert_allclose(interior, (2 * a * b + os_.C1) / (a * a + b * b + os_.C1), rtol=1e-11)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    xs = [rng.random((3, 9, 12)), rng.random((3, 7, 5))]
    ys = [np.clip(x + 0.1 * rng.standard_normal(x.shape), 0, 1) for x in xs]
    _, g = os_.loss_and_grad(xs, ys)
    h = 1e-6
    for v, x in enumerate(xs):
        for idx in [(0, 0, 0), (1, 4, 3), (2, x.shape[1] - 1, x.shape[2] - 1), (0, 3, 1)]:
            xp = [a.copy() for a in xs]
            xm = [a.copy() for a in xs]
            xp[v][idx] += h
            xm[v][idx] -= h
            fd = (os_.loss_and_grad(xp, ys)[0] - os_.loss_and_grad(xm, ys)[0]) / (2 * h)
            np.testing.assert_allclose(g[v][idx], fd, rtol=1e-6, atol=1e-12)


def test_sign_of_degradation():
    # blurring the target lowers SSIM: D grows with the noise added
    rng = np.random.default_rng(3)
    y = rng.random((3, 24, 24))
    ds = [os_.loss_and_grad([np.clip(y + s * rng.standard_normal(y.shape), 0, 1)], [y])[0]
          for s in (0.01, 0.05, 0.2)]
    assert 0 < ds[0] < ds[1] < ds[2] < 1

"""Pins of the FP64 Eq. 5 loss (oracle/loss.py): the paper-weighted worked
example of tests/golden/, central differences of its gradient, and the
invariances the loss is built to have."""
import os

import numpy as np
import pytest

from oracle import loss

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "eq5_two_pixels.txt")


def _fixture():
    rows = {}
    px = []
    with open(GOLDEN) as f:
        for line in f:
            words = line.split("#", 1)[0].split()
            if not words:
                continue
            vals = [float(x) for x in words[1:]]
            if words[0] == "pixel":
                px.append(vals)
            else:
                rows[words[0]] = vals
    px = np.array(px).T                      # (12, N)
    return px[0:3], px[3:6], px[6:9], px[9:12], rows


def test_worked_example_with_the_papers_weights():
    rgb, gt_rgb, nrm, gt_nrm, rows = _fixture()
    assert tuple(rows["weights"]) == loss.W_PAPER
    L, d_rgb, d_nrm = loss.eq5(rgb, nrm, gt_rgb, gt_nrm)
    assert L == pytest.approx(rows["loss"][0], abs=1e-14)
    np.testing.assert_allclose(d_nrm[:, 1], rows["d_normal_pixel1"], atol=1e-15)
    # the L1 term's gradient: sign / (3 N), zero where the colours agree
    np.testing.assert_array_equal(d_rgb[:, 0], np.array([1, 0, -1]) / 6)
    np.testing.assert_array_equal(d_rgb[:, 1], 0)


def _random(seed, N=64):
    rng = np.random.default_rng(seed)
    rgb, gt_rgb = rng.random((3, N)), rng.random((3, N))
    nrm = rng.standard_normal((3, N)) * 0.7
    gt = rng.standard_normal((3, N))
    gt /= np.linalg.norm(gt, axis=0)
    gt[:, rng.random(N) < 0.2] = 0.0         # background pixels
    return rgb, nrm, gt_rgb, gt


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_gradient_matches_central_differences(seed):
    rgb, nrm, gt_rgb, gt = _random(seed)
    L, d_rgb, d_nrm = loss.eq5(rgb, nrm, gt_rgb, gt)
    h = 1e-6
    for arr, grad in ((rgb, d_rgb), (nrm, d_nrm)):
        for idx in np.ndindex(*arr.shape):
            if arr is rgb and abs(rgb[idx] - gt_rgb[idx]) < 10 * h:
                continue                      # |x| at its kink
            p, m = arr.copy(), arr.copy()
            p[idx] += h
            m[idx] -= h
            args_p = (p, nrm) if arr is rgb else (rgb, p)
            args_m = (m, nrm) if arr is rgb else (rgb, m)
            fd = (loss.eq5(args_p[0], args_p[1], gt_rgb, gt)[0] - loss.eq5(args_m[0], args_m[1], gt_rgb, gt)[0]) / (2 * h)
            assert fd == pytest.approx(grad[idx], rel=1e-5, abs=1e-8), idx


def test_normal_term_ignores_orientation_and_scale_of_agreement():
    rgb, nrm, gt_rgb, gt = _random(4)
    L = loss.eq5(rgb, nrm, gt_rgb, gt)[0]
    # flipping every rendered normal changes neither |n x n^| nor the min
    assert loss.eq5(rgb, -nrm, gt_rgb, gt)[0] == pytest.approx(L, rel=1e-14)
    # identical images and normals: zero loss and zero gradient
    L0, g0, n0 = loss.eq5(gt_rgb, gt, gt_rgb, gt)
    assert L0 == 0.0 and not g0.any() and not n0.any()
    # a rendered normal parallel to the truth has no cross term: only the
    # min term remains, w2 w3 | |n^| - 1 | per pixel for a unit truth
    fg = np.linalg.norm(gt, axis=0) > 0
    s = 1.7
    L1 = loss.eq5(gt_rgb[:, fg], s * gt[:, fg], gt_rgb[:, fg], gt[:, fg])[0]
    assert L1 == pytest.approx(10 * 0.1 * abs(s - 1), rel=1e-13)


def test_weights_scale_their_terms():
    rgb, nrm, gt_rgb, gt = _random(5)
    only_rgb = loss.eq5(rgb, nrm, gt_rgb, gt, w=(1.0, 0.0, 0.1))[0]
    assert only_rgb == pytest.approx(np.abs(rgb - gt_rgb).mean(), rel=1e-14)
    a = loss.eq5(rgb, nrm, gt_rgb, gt, w=(0.0, 1.0, 0.0))[0]
    cross = np.linalg.norm(np.cross(gt.T, nrm.T), axis=1).mean()
    assert a == pytest.approx(cross, rel=1e-13)

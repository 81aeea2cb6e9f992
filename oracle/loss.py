"""FP64 reference of the training loss of Eq. 5 (Sec. 3.3) and its gradient
with respect to the rendered images.  TEST INFRASTRUCTURE ONLY (see
oracle/__init__.py).

For rendered colours I^ and normals n^ against ground truth I and n:
    L   = w1 |I - I^|_1 + w2 L_n,
    L_n = |n x n^|_2 + w3 min(|n - n^|_2, |n + n^|_2),
with w1 = 1, w2 = 10, w3 = 0.1 as the paper states beside the equation.

Readings (the paper does not say how the norms are reduced over an image):
the L1 term is the mean of |I - I^| over every pixel and colour channel;
L_n is evaluated per pixel and averaged over the pixels; several views are
one image of all their pixels.  A background pixel has the zero normal as
ground truth, so its cross term vanishes and its min term is |n^|.  The
gradient of a norm at 0 and of |x| at 0 are taken as 0; where the two
branches of the min are equal, the |n - n^| branch is taken.
"""
from __future__ import annotations

import numpy as np

W_PAPER = (1.0, 10.0, 0.1)


def _cross(a, b):
    """Cross product of (3, N) arrays, column by column."""
    return np.stack([a[1] * b[2] - a[2] * b[1],
                     a[2] * b[0] - a[0] * b[2],
                     a[0] * b[1] - a[1] * b[0]])


def _norm(a):
    return np.sqrt((a * a).sum(0))


def eq5(rgb, nrm, gt_rgb, gt_nrm, w=W_PAPER):
    """Loss and gradient of Eq. 5.

    rgb, nrm: rendered colour and normal, (3, N) float64, N pixels of all
    views; gt_rgb, gt_nrm: the ground truth, same shape.  Returns
    ``(loss, d_rgb, d_nrm)`` with the gradients shaped like the inputs.
    """
    w1, w2, w3 = w
    rgb, nrm = np.asarray(rgb, np.float64), np.asarray(nrm, np.float64)
    gt_rgb, gt_nrm = np.asarray(gt_rgb, np.float64), np.asarray(gt_nrm, np.float64)
    N = rgb.shape[1]
    # colour term: mean absolute difference over the 3 N values
    diff = rgb - gt_rgb
    l_rgb = np.abs(diff).sum() / (3 * N)
    d_rgb = w1 * np.sign(diff) / (3 * N)
    # normal term, pixel by pixel
    c = _cross(gt_nrm, nrm)                  # n x n^
    c_len = _norm(c)
    minus, plus = nrm - gt_nrm, nrm + gt_nrm
    m_len, p_len = _norm(minus), _norm(plus)
    take_minus = m_len <= p_len
    near = np.where(take_minus, m_len, p_len)
    l_n = (c_len + w3 * near).sum() / N
    # d|n x n^| / dn^ = (c x n) / |c|; d|n^ -+ n| / dn^ = (n^ -+ n) / |n^ -+ n|
    safe_c = np.where(c_len > 0, c_len, 1.0)
    g_cross = np.where(c_len > 0, _cross(c, gt_nrm) / safe_c, 0.0)
    vec = np.where(take_minus, minus, plus)
    safe_n = np.where(near > 0, near, 1.0)
    g_near = np.where(near > 0, vec / safe_n, 0.0)
    d_nrm = w2 * (g_cross + w3 * g_near) / N
    return w1 * l_rgb + w2 * l_n, d_rgb, d_nrm

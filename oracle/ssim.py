"""FP64 reference of the SSIM term of an "L1 + SSIM" image loss.  TEST
INFRASTRUCTURE ONLY (see oracle/__init__.py).

Per channel, local statistics over an 11 x 11 Gaussian window (sigma 1.5,
normalised to sum 1, pixels outside the image taken as zero):
    mx = w * x, my = w * y, sxx = w * x^2 - mx^2, syy = w * y^2 - my^2,
    sxy = w * (x y) - mx my,
    SSIM = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sxx + syy + C2)),
with C1 = 0.01^2 and C2 = 0.03^2 (images in [0, 1]), and the loss term
D = 1 - mean SSIM over every pixel and channel of the views.  The gradient
with respect to the rendered image x is written out by the chain rule
through the window sums (the window is symmetric, so the adjoint of the
blur is the blur itself).
"""
from __future__ import annotations

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2
RADIUS = 5
SIGMA = 1.5


def window() -> np.ndarray:
    k = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    w = np.exp(-k * k / (2.0 * SIGMA * SIGMA))
    return w / w.sum()


def blur(img: np.ndarray) -> np.ndarray:
    """Zero-padded separable correlation of an (H, W) image with the window."""
    w = window()
    H, W = img.shape
    pad = np.zeros((H + 2 * RADIUS, W + 2 * RADIUS))
    pad[RADIUS:RADIUS + H, RADIUS:RADIUS + W] = img
    rows = sum(w[k] * pad[:, k:k + W] for k in range(2 * RADIUS + 1))          # (H + 2R, W)
    return sum(w[k] * rows[k:k + H, :] for k in range(2 * RADIUS + 1))          # (H, W)


def ssim_terms(x: np.ndarray, y: np.ndarray) -> dict:
    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    n1 = 2 * mx * my + C1
    n2 = 2 * sxy + C2
    d1 = mx * mx + my * my + C1
    d2 = sxx + syy + C2
    S = n1 * n2 / (d1 * d2)
    return dict(S=S, mx=mx, my=my, n1=n1, n2=n2, d1=d1, d2=d2)


def loss_and_grad(views_x: list, views_y: list) -> tuple:
    """D = 1 - mean SSIM over all views (each (3, H, W)) and dD/dx per view."""
    total = sum(x.size for x in views_x)
    ssum = 0.0
    grads = []
    for x, y in zip(views_x, views_y):
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        g = np.zeros_like(x)
        for c in range(x.shape[0]):
            t = ssim_terms(x[c], y[c])
            S = t["S"]
            ssum += S.sum()
            # partial derivatives of S with respect to mx, E[x^2], E[xy]
            dmx = S * (2 * t["my"] / t["n1"] - 2 * t["my"] / t["n2"] - 2 * t["mx"] / t["d1"] + 2 * t["mx"] / t["d2"])
            dexx = -S / t["d2"]
            dexy = 2 * S / t["n2"]
            g[c] = -(blur(dmx) + 2 * x[c] * blur(dexx) + y[c] * blur(dexy)) / total
        grads.append(g)
    return 1.0 - ssum / total, grads

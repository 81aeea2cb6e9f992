"""A second, independently written FP64 renderer used only to pin the oracle.

It is deliberately written differently from the C oracle: the rotation comes
from ``scipy.spatial.transform.Rotation`` (a library routine, scalar-last
quaternions), the 3D covariance is formed explicitly as R diag(s^2) R^T, the
screen covariance as J T Sigma T^T J^T (Eq. 4) with the 2x2 inverse from
``numpy.linalg.inv``, and compositing (Eq. 1-2) is vectorised over all pixels
with one Gaussian at a time in depth order.  It has the same readings as the
oracle (near cull, low-pass dilation, pixel centres at +0.5, 3-sigma box and
ellipse, alpha clamp, floor, transmittance cutoff).
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation


F32 = lambda x: float(np.float32(x))  # noqa: E731  (constants are fp32 inputs)


def brute_render(g, cam, lowpass=F32(0.3), k=3.0, alpha_floor=F32(1 / 255), alpha_max=F32(0.99),
                 t_min=F32(1e-4), bg=(0.0, 0.0, 0.0)):
    W, H = cam["width"], cam["height"]
    V = np.asarray(cam["viewmat"], np.float64)
    T, t = V[:, :3], V[:, 3]
    fx, fy, cx, cy = (float(np.float32(cam[s])) for s in ("fx", "fy", "cx", "cy"))
    near = float(np.float32(cam["near"]))
    mu = np.asarray(g["mean"], np.float64)
    n = len(mu)
    pc = mu @ T.T + t
    z32 = pc[:, 2].astype(np.float32)
    order = sorted(range(n), key=lambda i: (float(z32[i]), i))
    xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    Tr = np.ones((H, W))
    live = np.ones((H, W), bool)
    Cimg = np.zeros((3, H, W))
    Nimg = np.zeros((3, H, W))
    Dimg = np.zeros((H, W))
    for i in order:
        x, y, z = pc[i]
        q = np.asarray(g["quat"][i], np.float64)
        if not z > near or not np.any(q != 0):
            continue
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        S2 = np.diag(np.asarray(g["scale"][i], np.float64) ** 2)
        Sig = R @ S2 @ R.T
        J = np.array([[fx / z, 0.0, -x * fx / z ** 2], [0.0, fy / z, -y * fy / z ** 2]])
        Ss = J @ T @ Sig @ T.T @ J.T + lowpass * np.eye(2)
        if not np.linalg.det(Ss) > 0:
            continue
        Ci = np.linalg.inv(Ss)
        u, v = fx * x / z + cx, fy * y / z + cy
        ex, ey = k * np.sqrt(Ss[0, 0]), k * np.sqrt(Ss[1, 1])
        i0, i1 = max(0, np.ceil(u - ex - 0.5)), min(W - 1, np.floor(u + ex - 0.5))
        j0, j1 = max(0, np.ceil(v - ey - 0.5)), min(H - 1, np.floor(v + ey - 0.5))
        if i0 > i1 or j0 > j1:
            continue
        ii, jj = np.meshgrid(np.arange(W), np.arange(H))
        inrect = (ii >= i0) & (ii <= i1) & (jj >= j0) & (jj <= j1)
        dx, dy = xs - u, ys - v
        power = -0.5 * (Ci[0, 0] * dx * dx + Ci[1, 1] * dy * dy) - Ci[0, 1] * dx * dy
        a = np.minimum(alpha_max, float(g["opacity"][i]) * np.exp(power))
        use = live & inrect & (power >= -0.5 * k * k) & (a >= alpha_floor)
        Tn = Tr * (1.0 - a)
        stop = use & (Tn < t_min)
        live &= ~stop
        use &= ~stop
        w = np.where(use, a * Tr, 0.0)
        Cimg += w * np.asarray(g["rgb"][i], np.float64)[:, None, None]
        Nimg += w * np.asarray(g["normal"][i], np.float64)[:, None, None]
        Dimg += w * z
        Tr = np.where(use, Tn, Tr)
    rgb = Cimg + Tr * np.asarray(bg, np.float64)[:, None, None]
    return dict(rgb=rgb, normal=Nimg, depth=Dimg, alpha=1.0 - Tr)

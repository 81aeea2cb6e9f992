"""FP64 reference of the learned per-point estimator.  TEST INFRASTRUCTURE
ONLY (see oracle/__init__.py).

The paper's estimator predicts, per point, the Gaussian's scale, rotation
quaternion and opacity with a shared per-point MLP head (Sec. 3.1-3.2); the
sparse 3D UNet that feeds that head needs MinkowskiEngine and trained
weights, so the build replaces it with features from the point's 16 nearest
neighbours:

  features  for each neighbour j (in distance order):
              R^T (p_j - p_i) / r_i   and   c_j - c_i
            with R the canonical PCA frame of the point and r_i the distance
            to its 16th neighbour  (16 x 6 = 96 inputs)
  network   96 -> 64 -> 64 -> 64 (ReLU) -> 8, bf16 weights and activations
            (round to nearest even), fp32-or-better accumulation
  outputs   corrections of the PCA estimate in the PCA frame:
              s = s_pca * exp(clip(y0..2, -4, 4))
              q = q_pca (x) normalize((1 + y3, y4, y5, y6))
              o = sigmoid(logit(o_pca) + y7)
              normal = third column of R(q)
            A zero last layer reproduces the PCA estimate exactly.

The reference evaluates the matmuls in FP64 on the bf16-rounded operands
and re-rounds every hidden activation to bf16, as the tensor-core kernel
stores them; only the accumulation order differs from the GPU.
"""
from __future__ import annotations

import numpy as np

IN, HID, OUT, OUT_PAD = 96, 64, 8, 16
# blob: bf16 W1[64][96], W2[64][64], W3[64][64], W4[16][64] (rows 8-15
# zero), then fp32 b1[64], b2[64], b3[64], b4[16]
BF16_SHAPES = [("W1", (HID, IN)), ("W2", (HID, HID)), ("W3", (HID, HID)), ("W4", (OUT_PAD, HID))]
F32_SHAPES = [("b1", (HID,)), ("b2", (HID,)), ("b3", (HID,)), ("b4", (OUT_PAD,))]
N_BF16 = sum(int(np.prod(s)) for _, s in BF16_SHAPES)
N_F32 = sum(int(np.prod(s)) for _, s in F32_SHAPES)
BLOB_BYTES = 2 * N_BF16 + 4 * N_F32


def bf16_round(x) -> np.ndarray:
    """Round to bfloat16 (nearest even) through fp32; returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed: int = 0) -> dict:
    """He-style random hidden layers, zero last layer (net == PCA)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, (o, i) in BF16_SHAPES:
        p[name] = rng.standard_normal((o, i)) * np.sqrt(2.0 / i)
    p["W4"][:] = 0.0
    for name, shp in F32_SHAPES:
        p[name] = np.zeros(shp)
    return p


def pack_blob(p: dict) -> np.ndarray:
    """Byte blob (uint8) in the layout above."""
    parts = []
    for name, shp in BF16_SHAPES:
        w = np.zeros(shp, np.float32)
        src = np.asarray(p[name], np.float64)
        w[: src.shape[0], : src.shape[1]] = src
        u = bf16_round(w).astype(np.float32).view(np.uint32) >> 16
        parts.append(u.astype(np.uint16).reshape(-1).view(np.uint8))
    for name, shp in F32_SHAPES:
        b = np.zeros(shp, np.float32)
        src = np.asarray(p[name], np.float64)
        b[: src.shape[0]] = src
        parts.append(b.view(np.uint8))
    return np.concatenate(parts)


def unpack_blob(blob: np.ndarray) -> dict:
    blob = np.asarray(blob, np.uint8)
    p, off = {}, 0
    for name, shp in BF16_SHAPES:
        k = int(np.prod(shp))
        u = blob[off: off + 2 * k].view(np.uint16).astype(np.uint32) << 16
        p[name] = u.view(np.float32).astype(np.float64).reshape(shp)
        off += 2 * k
    for name, shp in F32_SHAPES:
        k = int(np.prod(shp))
        p[name] = blob[off: off + 4 * k].view(np.float32).astype(np.float64).reshape(shp)
        off += 4 * k
    return p


def quat_to_rot(q) -> np.ndarray:
    q = np.asarray(q, np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = np.moveaxis(q, -1, 0)
    return np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                     np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                     np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def features(xyz, rgb, idx, quat) -> np.ndarray:
    """(n, 96) FP64 features: per neighbour R^T (p_j - p_i) / r_i, c_j - c_i."""
    P = np.asarray(xyz, np.float64)
    Cc = np.asarray(rgb, np.float64)
    R = quat_to_rot(quat)
    d = P[idx] - P[:, None, :]                       # (n, 16, 3)
    r = np.sqrt((d[:, 15] ** 2).sum(-1))
    loc = np.einsum("nki,nij->nkj", d, R) / np.maximum(r, 1e-12)[:, None, None]
    col = Cc[idx] - Cc[:, None, :]
    return np.concatenate([loc, col], -1).reshape(len(P), IN)


def forward(p: dict, x) -> np.ndarray:
    """(n, 8) raw outputs; operands bf16-rounded, hidden activations
    re-rounded to bf16, matmuls in FP64."""
    h = bf16_round(x)
    for w, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        h = bf16_round(np.maximum(h @ bf16_round(p[w]).T + np.asarray(p[b], np.float32), 0.0))
    y = h @ bf16_round(p["W4"]).T + np.asarray(p["b4"], np.float32)
    return y[:, :OUT]


def apply_corrections(scale_pca, quat_pca, opacity_pca, y) -> dict:
    y = np.asarray(y, np.float64)
    s = np.asarray(scale_pca, np.float64) * np.exp(np.clip(y[:, 0:3], -4.0, 4.0))
    dq = np.stack([1.0 + y[:, 3], y[:, 4], y[:, 5], y[:, 6]], 1)
    dq /= np.linalg.norm(dq, axis=1, keepdims=True)
    a = np.asarray(quat_pca, np.float64)
    a = a / np.linalg.norm(a, axis=1, keepdims=True)
    w1, x1, y1, z1 = a.T
    w2, x2, y2, z2 = dq.T
    q = np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                  w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)
    o0 = np.asarray(opacity_pca, np.float64)
    o = 1.0 / (1.0 + np.exp(-(np.log(o0 / (1.0 - o0)) + y[:, 7])))
    normal = quat_to_rot(q)[:, :, 2]
    return dict(scale=s, quat=q, opacity=o, normal=normal)


def estimate(xyz, rgb, p: dict, opacity: float = 0.9) -> dict:
    """Oracle of p2e_estimate mode 1: kNN-PCA, features, network, corrections."""
    from . import knn, pca
    idx, _ = knn(xyz)
    e = pca(xyz, idx)
    y = forward(p, features(xyz, rgb, idx, e["quat"]))
    out = apply_corrections(e["scale"], e["quat"], np.full(len(xyz), opacity), y)
    out.update(idx=idx, pca=e, y=y)
    return out


def _ident(x):
    return np.asarray(x, np.float64)


def loss_grad_params(p: dict, x, scale_pca, quat_pca, opacity_pca, up: dict, rounding: bool = True) -> dict:
    """Exact gradient of L = sum(up_scale * s) + sum(up_quat * q) +
    sum(up_opacity * o) + sum(up_normal * normal) with respect to the
    network's parameters, the outputs s, q, o, normal being those of
    :func:`apply_corrections` on the network's raw outputs.

    ``rounding=True`` rounds operands and hidden activations to bf16 as the
    tensor-core forward does (the rounding is held fixed, i.e. treated as
    the identity in the derivative); ``rounding=False`` is the plain FP64
    network, whose gradient the finite-difference pin checks.
    Returns gradients keyed like the parameters (W4, b4 with 16 rows).
    """
    r = bf16_round if rounding else _ident
    W = {k: r(p[k]) for k in ("W1", "W2", "W3", "W4")}
    b = {k: np.asarray(p[k], np.float32 if rounding else np.float64).astype(np.float64)
         for k in ("b1", "b2", "b3", "b4")}
    h0 = r(x)
    a1 = h0 @ W["W1"].T + b["b1"]
    h1 = r(np.maximum(a1, 0))
    a2 = h1 @ W["W2"].T + b["b2"]
    h2 = r(np.maximum(a2, 0))
    a3 = h2 @ W["W3"].T + b["b3"]
    h3 = r(np.maximum(a3, 0))
    y = (h3 @ W["W4"].T + b["b4"])[:, :OUT]
    n = len(y)
    # ---- output mapping backward
    s0 = np.asarray(scale_pca, np.float64)
    q0 = np.asarray(quat_pca, np.float64)
    q0 = q0 / np.linalg.norm(q0, axis=1, keepdims=True)
    dy = np.zeros((n, OUT))
    inside = (y[:, 0:3] > -4.0) & (y[:, 0:3] < 4.0)
    dy[:, 0:3] = np.where(inside, up["scale"] * s0 * np.exp(np.clip(y[:, 0:3], -4, 4)), 0.0)
    dq = np.stack([1.0 + y[:, 3], y[:, 4], y[:, 5], y[:, 6]], 1)
    dn = np.linalg.norm(dq, axis=1, keepdims=True)
    dh = dq / dn
    a0, a1_, a2_, a3_ = q0.T
    # q = L(q0) dh with L the left Hamilton product matrix
    L = np.stack([np.stack([a0, -a1_, -a2_, -a3_], 1), np.stack([a1_, a0, -a3_, a2_], 1),
                  np.stack([a2_, a3_, a0, -a1_], 1), np.stack([a3_, -a2_, a1_, a0], 1)], 1)
    qf = np.einsum("nij,nj->ni", L, dh)
    Wq, Xq, Yq, Zq = qf.T
    gn = np.asarray(up["normal"], np.float64)
    gq = np.asarray(up["quat"], np.float64).copy()
    gq[:, 0] += 2 * Yq * gn[:, 0] - 2 * Xq * gn[:, 1]
    gq[:, 1] += 2 * Zq * gn[:, 0] - 2 * Wq * gn[:, 1] - 4 * Xq * gn[:, 2]
    gq[:, 2] += 2 * Wq * gn[:, 0] + 2 * Zq * gn[:, 1] - 4 * Yq * gn[:, 2]
    gq[:, 3] += 2 * Xq * gn[:, 0] + 2 * Yq * gn[:, 1]
    gh = np.einsum("nji,nj->ni", L, gq)
    dy[:, 3:7] = (gh - dh * (dh * gh).sum(1, keepdims=True)) / dn
    o0 = np.asarray(opacity_pca, np.float64)
    o = 1.0 / (1.0 + np.exp(-(np.log(o0 / (1 - o0)) + y[:, 7])))
    dy[:, 7] = up["opacity"] * o * (1 - o)
    # ---- layers
    g = {}
    dyp = np.zeros((n, OUT_PAD))
    dyp[:, :OUT] = dy
    g["W4"] = dyp.T @ h3
    g["b4"] = dyp.sum(0)
    d3 = (dyp @ W["W4"]) * (a3 > 0)
    g["W3"], g["b3"] = d3.T @ h2, d3.sum(0)
    d2 = (d3 @ W["W3"]) * (a2 > 0)
    g["W2"], g["b2"] = d2.T @ h1, d2.sum(0)
    d1 = (d2 @ W["W2"]) * (a1 > 0)
    g["W1"], g["b1"] = d1.T @ h0, d1.sum(0)
    return g


def linear_outputs(p: dict, x, scale_pca, quat_pca, opacity_pca, up: dict) -> float:
    """The scalar whose gradient :func:`loss_grad_params` returns, with the
    plain FP64 network (for finite differences)."""
    h = np.asarray(x, np.float64)
    for w, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        h = np.maximum(h @ np.asarray(p[w], np.float64).T + np.asarray(p[b], np.float64), 0)
    y = (h @ np.asarray(p["W4"], np.float64).T + np.asarray(p["b4"], np.float64))[:, :OUT]
    out = apply_corrections(scale_pca, quat_pca, opacity_pca, y)
    return float((up["scale"] * out["scale"]).sum() + (up["quat"] * out["quat"]).sum() +
                 (up["opacity"] * out["opacity"]).sum() + (up["normal"] * out["normal"]).sum())


def splat_area_loss(scale, ref_scale, weight: float):
    """The rendering-cost term of the training loss (an option of this
    implementation, not the paper's): A = weight * mean_i (s_i0 s_i1) /
    (r_i0 r_i1) over the points, the footprint of each estimated splat's two
    largest axes relative to the reference estimate's; points whose
    reference area is not positive and finite count in the mean's n but add
    nothing.  Returns (A, dA/ds) with dA/ds of shape (n, 3) (zero for s2)."""
    s = np.asarray(scale, np.float64)[:, :3]
    r = np.asarray(ref_scale, np.float64)[:, :3]
    n = len(s)
    ra = r[:, 0] * r[:, 1]
    ok = np.isfinite(ra) & (ra > 0)
    g = np.zeros(n)
    g[ok] = s[ok, 0] * s[ok, 1] / ra[ok]
    d = np.zeros((n, 3))
    d[ok, 0] = weight / n * s[ok, 1] / ra[ok]
    d[ok, 1] = weight / n * s[ok, 0] / ra[ok]
    return weight * g.sum() / n, d

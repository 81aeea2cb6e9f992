"""FP64 CPU oracle of the splatting renderer and the point estimators.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports this
module; only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may call it.  It shares no code with the CUDA path; the only
module both sides use is ``scenes`` (seeded inputs, no method arithmetic).

What each function follows (paper sections of arXiv 2409.16504):

* :func:`project`       -- Sec. 3.1, Eq. 3-4 (EWA projection, 3-sigma bound)
* :func:`bin_keys`      -- Sec. 3.1 depth ordering, written as the
  (tile | depth) key list and its stable sort
* :func:`render`        -- Sec. 3.1, Eq. 1-2 (front-to-back alpha blending of
  colour, normal and depth)
* :mod:`oracle.grad`    -- exact derivative of :func:`render` (the
  differentiable splatting of Sec. 1 and 3.3)
* :mod:`oracle.estimate` -- kNN-PCA covariance estimate (the local
  covariance prior of Sec. 2.1) and the per-point MLP reference
* :mod:`oracle.raycast` -- exact ground-truth views of the analytic scenes
  (replaces the mesh rasterisation of Sec. 3.3)
* :mod:`oracle.loss`    -- the training loss of Eq. 5 (Sec. 3.3) and its
  gradient; :mod:`oracle.ssim` the SSIM term added to it
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "p2e_oracle.c"), os.path.join(_HERE, "knn_pca.c"),
         os.path.join(_HERE, "raycast.c")]
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

# Renderer constants are fp32 in the C ABI; the defaults are held at their
# fp32 values so that every consumer sees the same numbers.
DEFAULT_CFG = dict(tile=16, alpha_floor=float(np.float32(1.0 / 255.0)),
                   alpha_max=float(np.float32(0.99)), t_min=float(np.float32(1e-4)),
                   lowpass=float(np.float32(0.3)), sigma_mult=3.0, bg=(0.0, 0.0, 0.0))
# Knife-edge flag half-widths (power at the 3-sigma boundary, alpha at the
# floor, transmittance at the cutoff); pixels within them are reported, not
# compared, because fp32 and fp64 may take the discrete decision differently.
DEFAULT_FLAGS = dict(flag_power=1e-4, flag_alpha=1e-6, flag_t=1e-7)


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(s) for s in _SRCS)
    if force or stale:
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-fno-fast-math", "-o", _LIB + ".tmp", *_SRCS, "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.or_emit_keys.restype = C.c_int64
            _lib.or_num_threads.restype = C.c_int
    return _lib


def _f32(x) -> float:
    """Renderer constants are fp32 inputs; the oracle widens them exactly."""
    return float(np.float32(x))


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def cam_floats(cam: dict) -> np.ndarray:
    v = np.asarray(cam["viewmat"], np.float32).reshape(12)
    return np.concatenate([v, np.array([cam["fx"], cam["fy"], cam["cx"], cam["cy"],
                                        cam["near"]], np.float32)]).astype(np.float32)


def num_threads() -> int:
    return int(lib().or_num_threads())


def project(g: dict, cam: dict, cfg: dict | None = None) -> dict:
    """R1-R4 for every Gaussian of ``g`` under camera ``cam`` (Eq. 3-4)."""
    cfg = {**DEFAULT_CFG, **(cfg or {})}
    n = len(g["mean"])
    mean = np.ascontiguousarray(g["mean"], np.float32)
    scale = np.ascontiguousarray(g["scale"], np.float32)
    quat = np.ascontiguousarray(g["quat"], np.float32)
    out = dict(
        vis=np.zeros(n, np.uint8), xyz=np.zeros((n, 3)), uv=np.zeros((n, 2)),
        cov2=np.zeros((n, 3)), conic=np.zeros((n, 3)), prect=np.zeros((n, 4), np.int32),
        trect=np.zeros((n, 4), np.int32), ntiles=np.zeros(n, np.int32),
        zkey=np.zeros(n, np.float32))
    cf = cam_floats(cam)
    lib().or_project(C.c_int64(n), _p(mean), _p(scale), _p(quat), _p(cf),
                     C.c_int(cam["width"]), C.c_int(cam["height"]),
                     C.c_double(_f32(cfg["lowpass"])), C.c_double(_f32(cfg["sigma_mult"])),
                     C.c_int(cfg["tile"]), _p(out["vis"]), _p(out["xyz"]), _p(out["uv"]),
                     _p(out["cov2"]), _p(out["conic"]), _p(out["prect"]), _p(out["trect"]),
                     _p(out["ntiles"]), _p(out["zkey"]))
    return out


def tiles_of(cam: dict, tile: int):
    tx = -(-cam["width"] // tile)
    ty = -(-cam["height"] // tile)
    return tx, ty


def bin_keys(projs: list, cams: list, cfg: dict | None = None):
    """R5: (tile | depth) keys of every view, stably sorted, and per-tile
    ranges.  View v's tile ids start at the sum of the tile counts of views
    before it.  Returns ``(keys u64[K], vals u32[K], ranges u32[tiles,2])``.
    """
    cfg = {**DEFAULT_CFG, **(cfg or {})}
    tile = cfg["tile"]
    K = int(sum(int(p["ntiles"].sum()) for p in projs))
    keys = np.zeros(max(K, 1), np.uint64)
    vals = np.zeros(max(K, 1), np.uint32)
    base = 0
    off = 0
    for p, cam in zip(projs, cams):
        tx, ty = tiles_of(cam, tile)
        n = len(p["ntiles"])
        off += lib().or_emit_keys(C.c_int64(n), _p(p["trect"]), _p(p["ntiles"]), _p(p["zkey"]),
                                  C.c_int(tx), C.c_int64(base), _p(keys), _p(vals),
                                  C.c_int64(off))
        base += tx * ty
    assert off == K
    ranges = np.zeros((base, 2), np.uint32)
    lib().or_sort_ranges(C.c_int64(K), _p(keys), _p(vals), C.c_int64(base), _p(ranges))
    return keys[:K], vals[:K], ranges


def render(g: dict, cam: dict, cfg: dict | None = None, brute: bool = False,
           proj: dict | None = None, flags: dict | None = None) -> dict:
    """R6-R7 (Eq. 1-2): the FP64 image of one view.

    Returns dict with ``rgb (3,H,W)``, ``normal (3,H,W)``, ``depth (H,W)``,
    ``alpha (H,W)`` (float64), ``ncontrib``, ``last`` (Gaussian index of the
    last contributor, -1 if none) and ``flag`` (knife-edge pixels).
    """
    cfg = {**DEFAULT_CFG, **(cfg or {})}
    fl = {**DEFAULT_FLAGS, **(flags or {})}
    if proj is None:
        proj = project(g, cam, cfg)
    n = len(g["mean"])
    W, H = cam["width"], cam["height"]
    img = np.zeros((8, H, W))
    ncontrib = np.zeros((H, W), np.int32)
    last = np.zeros((H, W), np.int32)
    flag = np.zeros((H, W), np.uint8)
    params = np.array([_f32(cfg["alpha_floor"]), _f32(cfg["alpha_max"]), _f32(cfg["t_min"]),
                       _f32(cfg["sigma_mult"]), *[_f32(b) for b in cfg["bg"]],
                       fl["flag_power"], fl["flag_alpha"], fl["flag_t"]], np.float64)
    opac = np.ascontiguousarray(g["opacity"], np.float32)
    rgb = np.ascontiguousarray(g["rgb"], np.float32)
    nrm = np.ascontiguousarray(g["normal"], np.float32)
    lib().or_render(C.c_int64(n), C.c_int(W), C.c_int(H), _p(proj["vis"]), _p(proj["xyz"]),
                    _p(proj["uv"]), _p(proj["conic"]), _p(proj["prect"]), _p(proj["zkey"]),
                    _p(opac), _p(rgb), _p(nrm), _p(params), C.c_int(1 if brute else 0),
                    _p(img), _p(ncontrib), _p(last), _p(flag))
    return dict(rgb=img[0:3], normal=img[3:6], depth=img[6], alpha=img[7],
                ncontrib=ncontrib, last=last, flag=flag.astype(bool), proj=proj)


GRAD_KEYS = ("mean", "scale", "quat", "opacity", "rgb", "normal")


def render_grad(g: dict, cams: list, up: list, cfg: dict | None = None) -> dict:
    """R8: exact FP64 gradient of L = sum_v <up_v, images_v> with respect to
    the raw inputs (mean, scale, quaternion, opacity, rgb, normal), every
    discrete decision held fixed.  ``up[v]`` is an (8, H, W) array of the
    upstream weights of view v: rgb(3), normal(3), depth, alpha."""
    cfg = {**DEFAULT_CFG, **(cfg or {})}
    n = len(g["mean"])
    mean = np.ascontiguousarray(g["mean"], np.float32)
    scale = np.ascontiguousarray(g["scale"], np.float32)
    quat = np.ascontiguousarray(g["quat"], np.float32)
    opac = np.ascontiguousarray(g["opacity"], np.float32)
    rgb = np.ascontiguousarray(g["rgb"], np.float32)
    nrm = np.ascontiguousarray(g["normal"], np.float32)
    out = dict(mean=np.zeros((n, 3)), scale=np.zeros((n, 3)), quat=np.zeros((n, 4)),
               opacity=np.zeros(n), rgb=np.zeros((n, 3)), normal=np.zeros((n, 3)))
    params = np.array([_f32(cfg["alpha_floor"]), _f32(cfg["alpha_max"]), _f32(cfg["t_min"]),
                       _f32(cfg["sigma_mult"]), *[_f32(b) for b in cfg["bg"]], 0, 0, 0], np.float64)
    for cam, u in zip(cams, up):
        p = project(g, cam, cfg)
        g2d = np.zeros((n, 13))
        upc = np.ascontiguousarray(u, np.float64)
        lib().or_render_grad(C.c_int64(n), C.c_int(cam["width"]), C.c_int(cam["height"]),
                             _p(p["vis"]), _p(p["xyz"]), _p(p["uv"]), _p(p["conic"]),
                             _p(p["prect"]), _p(p["zkey"]), _p(opac), _p(rgb), _p(nrm),
                             _p(params), _p(upc), _p(g2d))
        cf = cam_floats(cam)
        lib().or_project_grad(C.c_int64(n), _p(mean), _p(scale), _p(quat), _p(cf),
                              C.c_int(cam["width"]), C.c_int(cam["height"]),
                              C.c_double(_f32(cfg["lowpass"])), _p(p["vis"]), _p(g2d),
                              _p(out["mean"]), _p(out["scale"]), _p(out["quat"]),
                              _p(out["opacity"]), _p(out["rgb"]), _p(out["normal"]))
    return out


def linear_loss(g: dict, cams: list, up: list, cfg: dict | None = None):
    """L = sum_v <up_v, images_v> and the per-view renders (for finite
    differences of :func:`render_grad`)."""
    tot = 0.0
    rs = []
    for cam, u in zip(cams, up):
        r = render(g, cam, cfg)
        img = np.concatenate([r["rgb"], r["normal"], r["depth"][None], r["alpha"][None]])
        tot += float((img * u).sum())
        rs.append(r)
    return tot, rs


# ---------------------------------------------------------------- kNN-PCA
def knn(xyz) -> tuple:
    """Exact 16 nearest other points (FP64 distance, ties by index).
    Returns ``(idx int64 (n,16), d2 float64 (n,16))``."""
    p = np.ascontiguousarray(xyz, np.float32)
    n = len(p)
    idx = np.zeros((n, 16), np.int64)
    d2 = np.zeros((n, 16))
    lib().or_knn(C.c_int64(n), _p(p), _p(idx), _p(d2))
    return idx, d2


def pca(xyz, idx, kappa: float = 1.0, flat: float = 0.1) -> dict:
    """Neighbour covariance, its eigen-decomposition and the Gaussian it
    implies (scale, unit quaternion, normal)."""
    p = np.ascontiguousarray(xyz, np.float32)
    n = len(p)
    ix = np.ascontiguousarray(idx, np.int64)
    out = dict(cov=np.zeros((n, 6)), lam=np.zeros((n, 3)), scale=np.zeros((n, 3)),
               quat=np.zeros((n, 4)), normal=np.zeros((n, 3)))
    lib().or_pca(C.c_int64(n), _p(p), _p(ix), C.c_double(kappa), C.c_double(flat), _p(out["cov"]),
                 _p(out["lam"]), _p(out["scale"]), _p(out["quat"]), _p(out["normal"]))
    return out


def estimate_pca(xyz, rgb, opacity: float = 0.9, kappa: float = 1.0, flat: float = 0.1) -> dict:
    """kNN-PCA Gaussian set of a coloured point cloud (fp32, renderer input)."""
    idx, _ = knn(xyz)
    e = pca(xyz, idx, kappa, flat)
    n = len(xyz)
    return dict(mean=np.asarray(xyz, np.float32), scale=e["scale"].astype(np.float32),
                quat=e["quat"].astype(np.float32), opacity=np.full(n, opacity, np.float32),
                rgb=np.asarray(rgb, np.float32), normal=e["normal"].astype(np.float32))


def mean_nn_distance(xyz) -> float:
    """The cloud's average point distance d: the mean over points of the
    distance to the nearest other point (FP64)."""
    _, d2 = knn(xyz)
    return float(np.sqrt(d2[:, 0]).mean())


def estimate_global(xyz, rgb, sigma_rel: float, opacity: float = 0.9) -> dict:
    """The comparison estimator of Sec. 4.1 (one isotropic Gaussian size for
    the whole cloud, from the global point density): scale sigma_rel * d
    on every axis, identity rotation; the normal is the kNN-PCA normal."""
    idx, d2 = knn(xyz)
    e = pca(xyz, idx)
    n = len(xyz)
    d = float(np.sqrt(d2[:, 0]).mean())
    return dict(mean=np.asarray(xyz, np.float32), scale=np.full((n, 3), sigma_rel * d, np.float32),
                quat=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)), opacity=np.full(n, opacity, np.float32),
                rgb=np.asarray(rgb, np.float32), normal=e["normal"].astype(np.float32), dbar=d)


def relight(rgb, normal, alpha, lights, ambient: float, bg=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Late shading of one view from its rendered normal image (Sec. 3.1: a
    pixel shader on the normal map), Lambertian directional lights plus
    ambient, in FP64: C = rgb - (1 - alpha) bg, n^ = N / |N|,
    s = ambient + sum_l I_l max(0, n^ . l^_l) (s = 1 where |N| <= 1e-12),
    out = C s + (1 - alpha) bg.  rgb, normal: (3, H, W); alpha: (H, W)."""
    rgb = np.asarray(rgb, np.float64)
    N = np.asarray(normal, np.float64)
    a = np.asarray(alpha, np.float64)
    bgv = np.asarray(bg, np.float64)[:, None, None]
    C = rgb - (1.0 - a)[None] * bgv
    norm = np.sqrt((N * N).sum(0))
    has = norm > 1e-12
    nh = np.where(has[None], N / np.where(has, norm, 1.0)[None], 0.0)
    s = np.full(a.shape, float(ambient))
    for lx, ly, lz, inten in lights:
        l = np.array([lx, ly, lz], np.float64)
        l = l / np.linalg.norm(l)
        s = s + inten * np.maximum(0.0, np.einsum("chw,c->hw", nh, l))
    s = np.where(has, s, 1.0)
    return C * s[None] + (1.0 - a)[None] * bgv


def point_raster(xyz, rgb, cam: dict, bg=(0.0, 0.0, 0.0)) -> dict:
    """The point-rasterisation baseline of Sec. 4.1 ("OpenGL": each point a
    1-pixel square with a depth test).  A point covers the pixel
    (floor(u), floor(v)) containing its projection, computed in fp32 with
    every operation rounded in the order written:
    x = ((T00 px + T01 py) + T02 pz) + t0 (likewise y, z), u = fx (x / z) + cx,
    v = fy (y / z) + cy; it is drawn when z > near and the pixel lies in the
    image.  The nearest point wins (ties by the lower index).  Returns
    ``rgb (3,H,W)`` (bg where nothing is drawn), ``depth (H,W)`` (0 there)
    and ``winner (H,W)`` (point index, -1)."""
    f32 = np.float32
    p = np.asarray(xyz, f32)
    V = np.asarray(cam["viewmat"], f32).reshape(3, 4)
    W, H = int(cam["width"]), int(cam["height"])

    def row(r):
        return ((V[r, 0] * p[:, 0] + V[r, 1] * p[:, 1]) + V[r, 2] * p[:, 2]) + V[r, 3]

    x, y, z = row(0), row(1), row(2)
    near = f32(cam.get("near", 0.01))
    with np.errstate(divide="ignore", invalid="ignore"):
        u = f32(cam["fx"]) * (x / z) + f32(cam["cx"])
        v = f32(cam["fy"]) * (y / z) + f32(cam["cy"])
        ok = (z > near) & (z > 0) & (u >= 0) & (v >= 0) & (u < f32(W)) & (v < f32(H))
    idx = np.nonzero(ok)[0]
    pi = np.minimum(np.floor(u[idx]).astype(np.int64), W - 1)
    pj = np.minimum(np.floor(v[idx]).astype(np.int64), H - 1)
    pix = pj * W + pi
    order = np.lexsort((idx, z[idx], pix))          # by pixel, then depth, then index
    first = np.ones(len(order), bool)
    first[1:] = pix[order][1:] != pix[order][:-1]
    win = order[first]
    winner = np.full(H * W, -1, np.int64)
    winner[pix[win]] = idx[win]
    depth = np.zeros(H * W, f32)
    depth[pix[win]] = z[idx[win]]
    out = np.empty((3, H * W), f32)
    out[:] = np.asarray(bg, f32)[:, None]
    col = np.asarray(rgb, f32)
    out[:, pix[win]] = col[idx[win], :3].T
    return dict(rgb=out.reshape(3, H, W), depth=depth.reshape(H, W), winner=winner.reshape(H, W))


def sigma_of(scale, quat) -> np.ndarray:
    """Sigma = R diag(s^2) R^T for each row (quaternions normalised)."""
    q = np.asarray(quat, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
                  np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
                  np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], 1)
    s2 = np.asarray(scale, np.float64) ** 2
    return np.einsum("nij,nj,nkj->nik", R, s2, R)


# ---------------------------------------------------------------- ground truth
def prim_records(prims) -> np.ndarray:
    """Analytic primitives (scenes.Primitive) as the ray caster's records."""
    out = np.zeros((len(prims), 20))
    for k, p in enumerate(prims):
        if p.kind == "ell":
            out[k, 0] = 0
            out[k, 1:4], out[k, 4:7] = p.center, p.radii
            out[k, 7:16] = np.asarray(p.rot, np.float64).reshape(9)
        else:
            out[k, 0] = 1
            out[k, 1:4], out[k, 4:7], out[k, 7] = p.p0, p.p1, p.r
    return out


def raycast(prims, cam: dict, texture=None, bg=(0.0, 0.0, 0.0)) -> dict:
    """Exact ground-truth view: rgb (texture at the hit), outward normal,
    camera depth and coverage of one ray per pixel centre."""
    W, H = cam["width"], cam["height"]
    rec = np.ascontiguousarray(prim_records(prims))
    hit = np.zeros((H, W), np.uint8)
    depth = np.zeros((H, W))
    normal = np.zeros((H, W, 3))
    point = np.zeros((H, W, 3))
    cf = cam_floats(cam)
    lib().or_raycast(_p(cf), C.c_int(W), C.c_int(H), _p(rec), C.c_int(len(prims)), _p(hit),
                     _p(depth), _p(normal), _p(point))
    h = hit.astype(bool)
    rgb = np.zeros((H, W, 3)) + np.asarray(bg, np.float64)
    if texture is not None and h.any():
        rgb[h] = texture(point[h])
    return dict(hit=h, depth=depth, normal=normal.transpose(2, 0, 1), rgb=rgb.transpose(2, 0, 1),
                point=point)

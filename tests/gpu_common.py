"""Helpers shared by the GPU parity tests (seeded scenes, GPU render through
the C ABI, comparisons against the oracle)."""
from __future__ import annotations

import numpy as np
import torch

import oracle
import scenes

TOL = 1e-4  # max-abs per channel, fp32 GPU vs fp64 oracle


def cfg1_scene():
    g = scenes.sphere_cloud()
    cam = scenes.look_at_camera((0, 0, -3), (0, 0, 0), (0, -1, 0), 60, 128, 128)
    return g, cam


def random_scene(seed, n, W, H, cull_frac=0.05):
    """Random anisotropic Gaussians in front of a camera, a few of them
    culled (behind the near plane or with a zero quaternion)."""
    rng = np.random.default_rng(seed)
    cam = scenes.look_at_camera((0.1, -0.2, -2.0), (0, 0, 0), (0, 1, 0), 55, W, H)
    g = dict(mean=rng.uniform(-0.6, 0.6, (n, 3)).astype(np.float32),
             scale=np.exp(rng.uniform(np.log(0.002), np.log(0.05), (n, 3))).astype(np.float32),
             quat=rng.standard_normal((n, 4)).astype(np.float32),
             opacity=rng.uniform(0.05, 1.0, n).astype(np.float32),
             rgb=rng.random((n, 3)).astype(np.float32),
             normal=rng.standard_normal((n, 3)).astype(np.float32))
    k = int(cull_frac * n)
    if k:
        idx = rng.choice(n, size=2 * k, replace=False)
        g["mean"][idx[:k]] = (0.0, 0.0, -2.5)          # behind the camera
        g["quat"][idx[k:]] = 0.0                        # zero quaternion
    return g, cam


def humanoid_scene(n, W, H, seed=2):
    xyz, rgb, nrm, prims = scenes.humanoid_cloud(n, seed=seed)
    sp = scenes.mean_spacing(n, prims)
    g = scenes.surface_gaussians(xyz, nrm, rgb, 1.13 * sp, np.random.default_rng(seed))
    cam = scenes.sphere_camera(xyz.mean(0), 2.5, np.random.default_rng(seed), W, H)
    return g, cam


def gpu_render(g, cams, cfg=None, capacity=1 << 16):
    from paper_2409_16504_gb300 import GaussianSet, Renderer
    gs = GaussianSet.from_numpy(g)
    r = Renderer(cfg, capacity=capacity)
    out = r.render(gs, cams)
    torch.cuda.synchronize()
    return r, out


def gpu_proj_view(r, v, n):
    """Projected records of view v as numpy (rect as (tx0, tx1, ty0, ty1))."""
    sl = slice(v * n, (v + 1) * n)
    xy = r.proj.xy_depth[sl].cpu().numpy()
    co = r.proj.conic_op[sl].cpu().numpy()
    rect = (r.proj.rect[sl].cpu().numpy().astype(np.int32) & 0xFFFF)
    nt = r.proj.ntiles[sl].cpu().numpy().astype(np.int64)
    packed = xy[:, 3].view(np.uint32)
    iu = (packed & 0xFFFF).astype(np.uint16).view(np.int16).astype(np.float64)
    iv = (packed >> 16).astype(np.uint16).view(np.int16).astype(np.float64)
    uv = np.stack([iu + xy[:, 0], iv + xy[:, 1]], 1)
    return dict(uv=uv, zkey=xy[:, 2].copy(), conic=co[:, :3], prect=rect[:, [0, 2, 1, 3]], ntiles=nt)


# Knife-edge pixels (the oracle's flags: a splat's power within 1e-4 of the
# 3-sigma boundary, alpha within 1e-6 of the floor or T within 1e-7 of the
# cutoff) are excluded from the tolerance check because fp32 and fp64 may
# take the discrete decision differently there.  Their number is bounded:
# on the seeded test scenes it is 0-0.06 % of the pixels.
MAX_FLAG_FRAC = 1e-3


def compare_images(gpu: dict, orc: dict, tol=TOL, check_last=True, vals=None, ranges=None,
                   tile=16, tile_base=0, tiles_x=None, max_flag_frac=MAX_FLAG_FRAC,
                   max_flag_mismatch=None):
    """Element-wise comparison on unflagged pixels.  Returns the max error
    per plane, the number of flagged pixels and how many of those differ by
    more than ``tol`` (the decisions fp32 actually took differently);
    asserts the flagged fraction is at most ``max_flag_frac`` and, if given,
    the mismatching flagged pixels at most ``max_flag_mismatch``."""
    flag = orc["flag"]
    ok = ~flag
    errs = {}
    bad = np.zeros(flag.shape, bool)
    for key in ("rgb", "normal"):
        d = np.abs(gpu[key].cpu().numpy().astype(np.float64) - orc[key])
        bad |= (d > tol).any(0)
        d = d[:, ok]
        errs[key] = float(d.max()) if d.size else 0.0
    for key in ("depth", "alpha"):
        d = np.abs(gpu[key].cpu().numpy().astype(np.float64) - orc[key])
        bad |= d > tol
        d = d[ok]
        errs[key] = float(d.max()) if d.size else 0.0
    for key, e in errs.items():
        assert e <= tol, f"{key}: max abs error {e:.3g} > {tol}"
    nflag = int(flag.sum())
    nmis = int((bad & flag).sum())
    print(f"flagged pixels {nflag} of {flag.size} ({nflag / flag.size:.2e}); of them beyond {tol}: {nmis}")
    assert nflag <= max_flag_frac * flag.size, f"{nflag} flagged pixels of {flag.size}"
    if max_flag_mismatch is not None:
        assert nmis <= max_flag_mismatch, f"{nmis} flagged pixels beyond the tolerance"
    errs["flagged"] = nflag
    errs["flagged_mismatch"] = nmis
    if check_last and vals is not None:
        last = gpu["last"].cpu().numpy().astype(np.int64)
        H, W = last.shape
        jj, ii = np.nonzero(ok)
        tl = tile_base + (jj // tile) * tiles_x + (ii // tile)
        lg = last[jj, ii]
        got = np.where(lg > 0, vals[np.maximum(lg - 1, 0)].astype(np.int64), -1)
        # `last` is a position in the tile list; the Gaussian it names must be
        # the oracle's last contributor
        assert (got == orc["last"][jj, ii]).all()
        starts = ranges[tl, 0].astype(np.int64)
        ends = ranges[tl, 1].astype(np.int64)
        assert ((lg == 0) | ((lg > starts) & (lg <= ends))).all()
    return errs

"""End-to-end training of the learned per-point estimator (Sec. 3.3) through
the differentiable splatting, on the GPU, by libp2e's own kernels:

    estimate (kNN-PCA, then the tcgen05 network)  -> Gaussians
    render the views                               -> RGB, normal images
    loss of Eq. 5 against the ground-truth views   -> dL/dimages
    render backward                                -> dL/d(scale, quat, opacity, normal)
    network backward                               -> dL/dparameters
    Adam                                           -> parameters + bf16 weight blob

This module only drives those C-ABI calls and owns the buffers.  Training
scenes are seeded humanoid proxies with jittered sizes and poses; their
ground-truth views come from ``scenes.gt_views`` (exact ray casting of the
analytic surfaces, the stand-in for images rasterised from meshes).
"""
from __future__ import annotations

import argparse
import ctypes as C
import math
import os
import sys
import time

import numpy as np
import torch

from . import _lib, mlp
from ._lib import P2EGaussians, check
from .estimate import LEARNED, PCA, Estimator, cloud_tensors
from .render import DEFAULT_CONFIG, GaussianSet, Renderer, _ptr, _stream, p2e_render_backward

LOSS_W = (1.0, 10.0, 0.1)   # w1, w2, w3 of Eq. 5
ORDER = ("W1", "W2", "W3", "W4", "b1", "b2", "b3", "b4")


def flatten(params: dict) -> torch.Tensor:
    return torch.cat([params[k].reshape(-1).to(torch.float32) for k in ORDER]).contiguous()


def unflatten(theta: torch.Tensor) -> dict:
    out, off = {}, 0
    for k in ORDER:
        n = int(np.prod(mlp.SHAPES[k]))
        out[k] = theta[off: off + n].reshape(mlp.SHAPES[k]).clone()
        off += n
    return out


def scene_parts(seed: int, n_points: int, n_views: int, res: int, jitter: float = 0.15, degrade=None):
    """Host-side parts of a scene: (prims, xyz, rgb, cameras).  ``degrade``:
    None, ("quant", alpha) for a 10-bit voxelised input coarsened by alpha,
    or ("sub", beta) for a random beta-subset (the input augmentations of
    Sec. 3.3); the ground truth stays exact."""
    import scenes
    prims = scenes.humanoid_primitives(seed, jitter=jitter)
    xyz, rgb, _, _ = scenes.humanoid_cloud(n_points, seed=seed, prims=prims)
    if degrade is not None:
        kind, amount = degrade
        if kind == "quant":
            xyz, rgb = scenes.quantize_cloud(xyz, rgb, alpha=amount)
        elif kind == "sub":
            xyz, rgb = scenes.subsample_cloud(xyz, rgb, amount, seed + 11)
        else:
            raise ValueError(f"unknown degradation {kind}")
    rng = np.random.default_rng(seed + 7)
    center = xyz.mean(0)
    cams = [scenes.sphere_camera(center, 2.5, rng, res, res) for _ in range(n_views)]
    return prims, xyz, rgb, cams


class Scene:
    """A training / evaluation scene: cloud on the device, cameras, and the
    ground-truth RGB and normal images in the renderer's planar layout."""

    def __init__(self, seed: int, n_points: int, n_views: int, res: int, jitter: float = 0.15,
                 device="cuda", degrade=None, parts=None, gt=None):
        """``parts`` / ``gt``: precomputed scene_parts(...) and ground-truth
        views (e.g. ray cast in a process pool), else computed here."""
        import scenes
        prims, xyz, rgb, cams = parts or scene_parts(seed, n_points, n_views, res, jitter, degrade)
        self.cams = cams
        if gt is None:
            gt = scenes.gt_views(prims, cams)
        self.xyz, self.rgb = cloud_tensors(xyz, rgb, device)
        self.n = len(xyz)
        self.gt_rgb = torch.from_numpy(np.concatenate([g["rgb"].reshape(-1) for g in gt]).astype(np.float32)).to(device)
        self.gt_normal = torch.from_numpy(
            np.concatenate([g["normal"].reshape(-1) for g in gt]).astype(np.float32)).to(device)
        self.view_pixels = (C.c_int64 * len(cams))(*[int(c["width"]) * int(c["height"]) for c in cams])


    def degraded(self, degrade, seed: int = 0, device="cuda") -> "Scene":
        """The same views and ground truth with a degraded input cloud
        (("quant", alpha) or ("sub", beta), as the constructor)."""
        import copy

        import scenes
        xyz = self.xyz[:, :3].cpu().numpy()
        rgb = self.rgb[:, :3].cpu().numpy()
        kind, amount = degrade
        if kind == "quant":
            xyz, rgb = scenes.quantize_cloud(xyz, rgb, alpha=amount)
        elif kind == "sub":
            xyz, rgb = scenes.subsample_cloud(xyz, rgb, amount, seed)
        else:
            raise ValueError(f"unknown degradation {kind}")
        out = copy.copy(self)
        out.xyz, out.rgb = cloud_tensors(xyz, rgb, device)
        out.n = len(xyz)
        return out


def loss_ssim(rgb: torch.Tensor, gt_rgb: torch.Tensor, sizes: list, weight: float, loss_dev: torch.Tensor,
              d_rgb: torch.Tensor, scratch: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Adds weight x (1 - mean SSIM) of the rendered colour to ``loss_dev`` and
    its gradient to ``d_rgb`` (p2e_loss_ssim); ``sizes`` = [(H, W)] per view.
    Returns the scratch buffer (grown if needed) for reuse."""
    npix = sum(h * w for h, w in sizes)
    need = 96 * npix + 256
    if scratch is None or scratch.numel() < need:
        scratch = torch.empty(need, dtype=torch.uint8, device=rgb.device)
    hw = (C.c_int32 * (2 * len(sizes)))(*[v for h, w in sizes for v in (h, w)])
    sp = (scratch.data_ptr() + 255) & ~255
    check("p2e_loss_ssim", _lib.load().p2e_loss_ssim(_ptr(rgb), _ptr(gt_rgb), hw, len(sizes), C.c_float(weight),
                                                     _ptr(loss_dev), _ptr(d_rgb), C.c_void_p(sp), need - 256,
                                                     _stream(stream)))
    return scratch


class Trainer:
    def __init__(self, n_max: int, seed: int = 0, lr: float = 1e-3, cfg: dict | None = None, device="cuda",
                 params: dict | None = None, ssim_weight: float = 0.0, area_weight: float = 0.0):
        """``ssim_weight`` > 0 adds that weight times the SSIM term
        (p2e_loss_ssim) of the colour to the Eq. 5 loss; ``area_weight`` > 0
        adds that weight times the splats' mean footprint relative to the
        kNN-PCA splats' (p2e_loss_splat_area), a rendering-cost term."""
        self.device = device
        # 8-px tiles: the backward's time follows the longest tile list
        # (measured 2.2 vs 3.9 ms at 200K points x 8 views at 512^2)
        self.cfg = {**DEFAULT_CONFIG, "tile": 8, **(cfg or {})}
        self.theta = flatten(params if params is not None else mlp.init_params(seed, device)).to(device)
        assert self.theta.numel() == _lib.MLP_PARAMS
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.grad = torch.zeros_like(self.theta)
        self.blob = mlp.pack(unflatten(self.theta))
        self.lr = lr
        self.t = 0
        self.est = Estimator(n_max, device)
        self.loss_dev = torch.zeros(1, dtype=torch.float32, device=device)
        # buffers reused across steps (the renderer grows its key buffers
        # when a scene needs more)
        self.rend = Renderer(self.cfg, capacity=1 << 20, device=device)
        self.knn = torch.empty((n_max, 16), dtype=torch.int32, device=device)
        self.g_pca = GaussianSet.empty(n_max, device)
        self.g_net = GaussianSet.empty(n_max, device)
        self.ssim_weight = float(ssim_weight)
        self.area_weight = float(area_weight)
        self.ssim_scratch = None

    def params(self) -> dict:
        return unflatten(self.theta)

    def _forward(self, sc: Scene, learned: bool = True):
        if sc.n > self.knn.shape[0]:
            self.knn = torch.empty((sc.n, 16), dtype=torch.int32, device=self.device)
            self.g_pca = GaussianSet.empty(sc.n, self.device)
            self.g_net = GaussianSet.empty(sc.n, self.device)
        n = sc.n
        knn = self.knn[:n]
        view = lambda g: GaussianSet(g.mean_op[:n], g.scale[:n], g.quat[:n], g.rgb[:n], g.normal[:n])  # noqa: E731
        g_pca = self.est(sc.xyz, sc.rgb, mode=PCA, knn=knn, out=view(self.g_pca))
        g = self.est(sc.xyz, sc.rgb, mode=LEARNED, mlp_blob=self.blob, out=view(self.g_net)) if learned else g_pca
        r = self.rend
        img = r.render(g, sc.cams)
        return knn, g_pca, g, r, img

    def _loss(self, sc: Scene, img):
        d_rgb = torch.empty_like(img.rgb)
        d_nrm = torch.empty_like(img.normal)
        check("p2e_loss_eq5", _lib.load().p2e_loss_eq5(
            _ptr(img.rgb), _ptr(img.normal), _ptr(sc.gt_rgb), _ptr(sc.gt_normal), sc.view_pixels,
            len(sc.cams), *LOSS_W, _ptr(self.loss_dev), _ptr(d_rgb), _ptr(d_nrm), _stream()))
        if self.ssim_weight > 0:
            sizes = [(int(c["height"]), int(c["width"])) for c in sc.cams]
            self.ssim_scratch = loss_ssim(img.rgb, sc.gt_rgb, sizes, self.ssim_weight, self.loss_dev, d_rgb,
                                          self.ssim_scratch)
        return d_rgb, d_nrm

    def step(self, sc: Scene) -> float:
        knn, g_pca, g, r, img = self._forward(sc)
        d_rgb, d_nrm = self._loss(sc, img)
        d = p2e_render_backward(g, r.proj, r.bins, sc.cams, r.cfg, img.alpha, img.last, d_rgb=d_rgb,
                                d_normal=d_nrm)
        ps = g_pca.c_struct()
        lib = _lib.load()
        if self.area_weight > 0:
            check("p2e_loss_splat_area", lib.p2e_loss_splat_area(
                _ptr(g.scale), _ptr(g_pca.scale), sc.n, self.area_weight, _ptr(self.loss_dev), _ptr(d["scale"]),
                _stream()))
        check("p2e_mlp_backward", lib.p2e_mlp_backward(
            _ptr(sc.xyz), _ptr(sc.rgb), sc.n, _ptr(knn), C.byref(ps), _ptr(self.blob), _ptr(d["scale"]),
            _ptr(d["quat"]), _ptr(d["opacity"]), _ptr(d["normal"]), _ptr(self.grad), _stream()))
        self.t += 1
        check("p2e_adam", lib.p2e_adam(_ptr(self.theta), _ptr(self.grad), _ptr(self.m), _ptr(self.v),
                                       self.theta.numel(), self.lr, 0.9, 0.999, 1e-8, self.t,
                                       _ptr(self.blob), _stream()))
        return float(self.loss_dev.item())

    @torch.no_grad()
    def evaluate(self, sc: Scene, learned: bool = True) -> dict:
        """Eq. 5 loss and RGB PSNR (all pixels, images in [0, 1]) of one scene."""
        _, _, _, _, img = self._forward(sc, learned)
        self._loss(sc, img)
        mse = float(((img.rgb - sc.gt_rgb) ** 2).mean().item())
        return dict(loss=float(self.loss_dev.item()), psnr=10.0 * math.log10(1.0 / max(mse, 1e-12)))


def time_differentiation(points: int = 200_000, views: int = 8, res: int = 512, ssim_weight: float = 0.2,
                         reps: int = 5, seed: int = 3, device="cuda", tile: int = 8, probe=None) -> dict:
    """Forward and backward of the splatting at the differentiation scale:
    a ``points``-point humanoid (kNN-PCA Gaussians), ``views`` views at
    res x res, loss = Eq. 5 + ssim_weight x the SSIM term against the exact
    ray-cast views, gradients with respect to every Gaussian parameter.
    Median CUDA-event milliseconds of each phase over ``reps`` runs.
    ``probe`` (optional, with ``arm(i)`` / ``disarm()``) is armed around
    the backward of timed run i (a kernel probe of the library)."""
    sc = Scene(seed, points, views, res, device=device)
    tr = Trainer(points, ssim_weight=ssim_weight, device=device, cfg={"tile": tile})
    knn, g_pca, g, r, img = tr._forward(sc, learned=False)
    st = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    rows = []
    for it in range(reps + 2):
        e = [ev() for _ in range(4)]
        e[0].record(st)
        img = r.render(g, sc.cams, out=img, check=False)
        e[1].record(st)
        d_rgb, d_nrm = tr._loss(sc, img)
        e[2].record(st)
        if probe is not None and it >= 2:
            probe.arm(it - 2)
        d = p2e_render_backward(g, r.proj, r.bins, sc.cams, r.cfg, img.alpha, img.last, d_rgb=d_rgb,
                                d_normal=d_nrm)
        if probe is not None:
            probe.disarm()
        e[3].record(st)
        torch.cuda.synchronize()
        if it >= 2:
            rows.append([e[k].elapsed_time(e[k + 1]) for k in range(3)])
    med = np.median(np.array(rows), 0)
    finite = all(bool(torch.isfinite(v).all()) for v in d.values())
    return dict(points=points, views=views, res=res, tile=tile, ssim_weight=ssim_weight, keys=r.n_keys,
                pixels=views * res * res,
                render_ms=float(med[0]), loss_ms=float(med[1]), backward_ms=float(med[2]),
                total_ms=float(med.sum()), loss=float(tr.loss_dev.item()), gradients_finite=finite)


def main(argv=None):
    ap = argparse.ArgumentParser(description="train the learned per-point estimator")
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--scenes", type=int, default=48)
    ap.add_argument("--points", type=int, nargs="+", default=[100_000, 1_000_000],
                    help="points per training scene: one value, or a range drawn log-uniformly per scene")
    ap.add_argument("--views", type=int, default=4)
    ap.add_argument("--res", type=int, default=512)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval-scenes", type=int, default=4)
    ap.add_argument("--out", default=mlp.TRAINED)
    ap.add_argument("--ssim", type=float, default=0.0, help="weight of the SSIM term added to the Eq. 5 loss")
    ap.add_argument("--area", type=float, default=0.0,
                    help="weight of the splat-footprint term (rendering cost) added to the loss")
    ap.add_argument("--augment", type=float, default=0.0,
                    help="fraction of training scenes with degraded inputs (10-bit voxels coarsened by "
                         "alpha in [0.25, 1], or a beta in [0.125, 1] random subset)")
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    t0 = time.time()
    rng = np.random.default_rng(0)

    def degrade_of(s):
        if rng.random() >= a.augment:
            return None
        return ("quant", float(rng.uniform(0.25, 1.0))) if rng.random() < 0.5 else \
            ("sub", float(rng.uniform(0.125, 1.0)))
    lo, hi = (a.points[0], a.points[-1])
    npts = [int(round(math.exp(rng.uniform(math.log(lo), math.log(hi))))) if hi > lo else lo
            for _ in range(a.scenes)]
    parts = [scene_parts(1000 + s, npts[s], a.views, a.res, degrade=degrade_of(s)) for s in range(a.scenes)]
    held_parts = [scene_parts(2000 + s, int(math.sqrt(lo * hi)), 12, a.res) for s in range(a.eval_scenes)]
    # ground truth ray cast in a process pool before the first GPU call
    from .evaluate import ground_truth
    gts = ground_truth([(p[0], p[3]) for p in parts + held_parts])
    pool = [Scene(0, 0, 0, 0, parts=p, gt=g) for p, g in zip(parts, gts[:len(parts)])]
    held = [Scene(0, 0, 0, 0, parts=p, gt=g) for p, g in zip(held_parts, gts[len(parts):])]
    print(f"scenes ready in {time.time() - t0:.1f} s (points {min(npts)}..{max(npts)})", flush=True)
    tr = Trainer(max(npts + [len(p[1]) for p in held_parts]), lr=a.lr, ssim_weight=a.ssim, area_weight=a.area)
    before = [tr.evaluate(h, learned=False) for h in held]
    t1 = time.time()
    for it in range(a.steps):
        loss = tr.step(pool[it % len(pool)])
        if it % 50 == 0 or it == a.steps - 1:
            print(f"step {it:5d} loss {loss:.5f}", flush=True)
    torch.cuda.synchronize()
    dt = time.time() - t1
    after = [tr.evaluate(h, learned=True) for h in held]
    mlp.save(tr.params(), a.out)
    pca_psnr = float(np.mean([b["psnr"] for b in before]))
    net_psnr = float(np.mean([x["psnr"] for x in after]))
    print(f"trained {a.steps} steps in {dt:.1f} s ({1e3 * dt / a.steps:.1f} ms/step); held-out PSNR "
          f"kNN-PCA {pca_psnr:.2f} dB, learned {net_psnr:.2f} dB; loss {np.mean([b['loss'] for b in before]):.4f}"
          f" -> {np.mean([x['loss'] for x in after]):.4f}; saved {a.out}", flush=True)


if __name__ == "__main__":
    main()

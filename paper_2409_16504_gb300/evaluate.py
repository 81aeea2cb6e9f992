"""Rendering quality of the estimators against exact ground truth (the
comparison of Sec. 4.2, Table 1, on synthetic stand-ins for THuman 2.0).

Protocol (Sec. 4.2: views on a circle around the subject at 512 x 512,
PSNR against views of the ground-truth surface): held-out humanoid scenes
(seeds never used in training), 12 cameras on a horizontal circle around
the subject's centroid, RGB PSNR per view averaged over views and scenes.
Ground truth: exact ray casts of the analytic surfaces (``scenes.gt_views``,
the stand-in for views rasterised from meshes).  Methods, all rendered by
libp2e:

  learned     kNN-PCA + the shipped trained per-point network
  knn_pca     the closed-form kNN-PCA estimate
  global_1.2, global_1.5, global_1.7
              one isotropic size sigma_rel x the mean nearest-neighbour
              distance for the whole cloud (Sec. 4.1 "global parameters")
  point_raster
              1-pixel squares with a depth test (Sec. 4.1 "OpenGL")

PSNR over the whole view (RGB in [0, 1], black background on both sides).
``python -m paper_2409_16504_gb300.evaluate`` runs the full held-out set
(seeds 2000-2015) and the 800K-point, 1024 x 1024 frame of the benchmark.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

import numpy as np

METHODS = ("learned", "knn_pca", "global_1.2", "global_1.5", "global_1.7", "point_raster")


def _gt(args):
    prims, cams = args
    import scenes
    return scenes.gt_views(prims, cams)


def ground_truth(jobs: list, workers: int | None = None) -> list:
    """Ray-cast views for each (prims, cams) job, one view per task, in a
    process pool started with `spawn` (safe next to a CUDA context)."""
    flat = [(p, [c]) for p, cams in jobs for c in cams]
    workers = workers or max(1, min(len(flat), (os.cpu_count() or 2)))
    with mp.get_context("spawn").Pool(workers) as pool:
        views = pool.map(_gt, flat)
    out, k = [], 0
    for _, cams in jobs:
        out.append([views[k + i][0] for i in range(len(cams))])
        k += len(cams)
    return out


def psnr(img: np.ndarray, ref: np.ndarray) -> float:
    mse = float(((np.asarray(img, np.float64) - ref) ** 2).mean())
    return 10.0 * math.log10(1.0 / max(mse, 1e-12))


WEIGHTS = None  # path of the network's weights (None: the shipped ones)


def render_methods(xyz: np.ndarray, rgb: np.ndarray, cams: list, device="cuda") -> dict:
    """Planar RGB (3, H, W) of every view for every method."""
    import torch

    from . import mlp
    from .estimate import LEARNED, PCA, Estimator, cloud_tensors
    from .render import GaussianSet, Images, Renderer, point_raster
    n = len(xyz)
    cx, cc = cloud_tensors(xyz, rgb, device)
    est = Estimator(n, device)
    params = mlp.load_params(WEIGHTS or mlp.TRAINED, device)
    blob = None if params is None else mlp.pack(params)
    rend = Renderer(capacity=1 << 22, device=device)
    out = {}
    for m in METHODS:
        if m == "point_raster":
            img = point_raster(cx, cc, cams)
        else:
            gs = GaussianSet.empty(n, device)
            if m == "learned":
                if blob is None:
                    continue
                est(cx, cc, mode=LEARNED, mlp_blob=blob, out=gs)
            elif m == "knn_pca":
                est(cx, cc, mode=PCA, out=gs)
            else:
                est.global_(cx, cc, float(m.split("_")[1]), out=gs)
            est.check(n)
            img = Images(cams, device)
            rend.render(gs, cams, out=img)
        torch.cuda.synchronize()
        out[m] = [img.view(v)["rgb"].cpu().numpy() for v in range(len(cams))]
    return out


def evaluate_scenes(scenes_: list, gts: list, device="cuda") -> dict:
    """Mean per-view PSNR of every method over (xyz, rgb, cams) scenes."""
    per = {m: [] for m in METHODS}
    for (xyz, rgb, cams), gt in zip(scenes_, gts):
        imgs = render_methods(xyz, rgb, cams, device)
        for m, views in imgs.items():
            per[m].extend(psnr(v, g["rgb"]) for v, g in zip(views, gt))
    return {m: float(np.mean(v)) for m, v in per.items() if v}


def held_out(seeds=range(2000, 2016), points: int = 150_000, views: int = 12, res: int = 512,
             radius: float = 2.5, fov: float = 60.0, device="cuda") -> dict:
    """The held-out protocol: per seed a jittered humanoid (as the training
    scenes) of ``points`` points, ``views`` cameras on a horizontal circle."""
    import scenes
    sc, jobs = [], []
    for s in seeds:
        prims = scenes.humanoid_primitives(s, jitter=0.15)
        xyz, rgb, _, _ = scenes.humanoid_cloud(points, seed=s, prims=prims)
        cams = scenes.circle_cameras(xyz.mean(0), radius, views, res, res, fov_deg=fov)
        sc.append((xyz, rgb, cams))
        jobs.append((prims, cams))
    gts = ground_truth(jobs)
    res_ = evaluate_scenes(sc, gts, device)
    res_.update(scenes=len(sc), views=views, res=res, points=points)
    return res_


def bench_frame(points: int = 800_000, res: int = 1024, views: int = 8, seed: int = 2, device="cuda") -> dict:
    """The benchmark's frame: the 800K-point humanoid (seed 2), cameras drawn
    on the 2.5 m sphere as the benchmark draws them."""
    import scenes
    xyz, rgb, _, prims = scenes.humanoid_cloud(points, seed=seed)
    rng = np.random.default_rng(seed + 100)
    cams = [scenes.sphere_camera(xyz.mean(0), 2.5, rng, res, res) for _ in range(views)]
    gts = ground_truth([(prims, cams)])
    out = evaluate_scenes([(xyz, rgb, cams)], gts, device)
    out.update(views=views, res=res, points=points)
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="rendering quality of the estimators against exact ground truth")
    ap.add_argument("--seeds", type=int, default=16, help="held-out scenes (seeds 2000 ..)")
    ap.add_argument("--points", type=int, default=150_000)
    ap.add_argument("--res", type=int, default=512)
    ap.add_argument("--bench-views", type=int, default=8)
    ap.add_argument("--weights", default=None, help="network weights (.npz); default: the shipped ones")
    a = ap.parse_args(argv)
    global WEIGHTS
    WEIGHTS = a.weights
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    t0 = time.time()
    out = {"held_out": held_out(range(2000, 2000 + a.seeds), a.points, 12, a.res),
           "bench_frame": bench_frame(views=a.bench_views)}
    out["seconds"] = time.time() - t0
    print(json.dumps(out))


if __name__ == "__main__":
    main()

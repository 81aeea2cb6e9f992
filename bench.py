#!/usr/bin/env python
"""Frame-latency / throughput benchmark of the splatting path at 1024x1024.

Workload: 800K points on the humanoid proxy (12 analytic primitives, 1 m
tall, 1 mm position noise, smooth-noise colours), one 1024x1024 view per
frame from a camera drawn uniformly on a 2.5 m sphere (re-drawn every frame).

A step is one frame of the whole path on the device: estimation of the
Gaussians from the resident point cloud (kNN-PCA, or kNN-PCA + learned MLP)
followed by projection, key emission + radix sort + tile ranges, and
compositing.  Per step the L2 is flushed (a 256 MiB write) outside the
timed interval; each step is timed with CUDA events on the launching
stream.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "p50/p99 frame latency (ms) and Mpix/s at 1024², learned vs kNN-PCA path"
N_POINTS = 800_000
RES = 1024
SEED = 2


def workload_name(path: str) -> str:
    return {"render": "800K-point humanoid proxy, surface-aligned Gaussians, 1024x1024 render "
                      "(projection + binning + radix sort + compositing)",
            "pca": "800K-point humanoid proxy, kNN-PCA estimation + 1024x1024 render",
            "learned": "800K-point humanoid proxy, kNN-PCA + learned MLP estimation + 1024x1024 render"}[path]


def make_inputs():
    import scenes
    xyz, rgb, nrm, prims = scenes.humanoid_cloud(N_POINTS, seed=SEED)
    sp = scenes.mean_spacing(N_POINTS, prims)
    g = scenes.surface_gaussians(xyz, nrm, rgb, 1.13 * sp, np.random.default_rng(SEED))
    return xyz, rgb, g


def cameras(center, k, seed):
    import scenes
    rng = np.random.default_rng(seed)
    return [scenes.sphere_camera(center, 2.5, rng, RES, RES) for _ in range(k)]


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def cpu_baseline(budget_s: float = 12.0) -> dict:
    """The FP64 oracle on the host cores, on a bounded sample of frames."""
    import oracle
    xyz, rgb, g = make_inputs()
    cams = cameras(xyz.mean(0), 64, SEED + 1)
    t0 = time.perf_counter()
    frames = 0
    while frames < len(cams) and (time.perf_counter() - t0) < budget_s:
        p = oracle.project(g, cams[frames])
        oracle.bin_keys([p], [cams[frames]])
        oracle.render(g, cams[frames], proj=p)
        frames += 1
    dt = time.perf_counter() - t0
    return {"value": frames * RES * RES / dt / 1e6, "unit": "Mpix/s", "cores": oracle.num_threads(),
            "kind": "oracle", "ms_per_frame": 1e3 * dt / frames,
            "sample": f"{frames} frames of the render stage (project + bin + composite) on the "
                      f"surface-aligned Gaussian set, 1024x1024"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    t0 = time.perf_counter()
    import oracle
    xyz, rgb, g = make_inputs()
    cams = cameras(xyz.mean(0), args.warmup + args.steps, SEED + 1)
    times = []
    for i, cam in enumerate(cams):
        t = time.perf_counter()
        p = oracle.project(g, cam)
        oracle.bin_keys([p], [cam])
        oracle.render(g, cam, proj=p)
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
    tot = sum(times)
    val = args.steps * RES * RES / tot / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mpix/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "p50_ms": 1e3 * float(np.percentile(times, 50)), "p99_ms": 1e3 * float(np.percentile(times, 99)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name("render"), "points": N_POINTS,
                                            "resolution": RES},
            "cpu_baseline": {"value": val, "unit": "Mpix/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": f"{args.steps} frames after {args.warmup} warm-up"},
            "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default="render", choices=["render", "pca", "learned"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile", type=int, default=16, choices=[8, 16, 32])
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    from paper_2409_16504_gb300 import GaussianSet, Images, Renderer

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    xyz, rgb, g = make_inputs()
    center = xyz.mean(0)
    e_steps = max(3, min(args.steps, 50))
    cams = cameras(center, args.warmup + max(args.steps, e_steps), SEED + 100 + rank)
    gs = GaussianSet.from_numpy(g, dev)
    st = torch.cuda.current_stream()
    # capacity from a probe frame, with headroom for other viewpoints
    rend = Renderer({"tile": args.tile}, capacity=1 << 21, device=dev)
    probe = rend.render(gs, [cams[0]])
    rend.capacity = int(rend.n_keys * 1.6) + 4096
    rend.render(gs, [cams[0]])
    img = Images([cams[0]], dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def frame(cam):
        from paper_2409_16504_gb300.render import p2e_project, p2e_render, p2e_sort_bin
        e0, e1, e2, e3 = ev(), ev(), ev(), ev()
        e0.record(st)
        p2e_project(gs, [cam], rend.cfg, rend.proj)
        e1.record(st)
        p2e_sort_bin(rend.proj, gs.n, [cam], rend.cfg, rend.bins)
        e2.record(st)
        p2e_render(gs, rend.proj, rend.bins, [cam], rend.cfg, img.rgb, img.normal, img.depth,
                   img.alpha, img.last)
        e3.record(st)
        return e0, e1, e2, e3

    for i in range(args.warmup):
        flush.fill_(i & 0xFF)
        frame(cams[i])
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    recs = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        recs.append(frame(cams[args.warmup + i]))
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    stage = np.array([[a.elapsed_time(b), b.elapsed_time(c), c.elapsed_time(d)] for a, b, c, d in recs])
    frame_ms = stage.sum(1)
    tot_ms = float(frame_ms.sum())
    if world > 1:
        t = torch.tensor([tot_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
    value = world * args.steps * RES * RES / (tot_ms / 1e3) / 1e6

    # end to end through the public API with host buffers
    host = {k: getattr(gs, k).cpu().pin_memory() for k in ("mean_op", "scale", "quat", "rgb", "normal")}
    out_host = torch.empty((3 * RES * RES + 3 * RES * RES + RES * RES,), dtype=torch.float32).pin_memory()
    gd = GaussianSet.empty(gs.n, dev)
    h2d = sum(t.numel() * 4 for t in host.values())
    d2h = out_host.numel() * 4
    for w in range(2):
        for k, t in host.items():
            getattr(gd, k).copy_(t, non_blocking=True)
        rend.render(gd, [cams[w]], out=img, check=False)
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record(st)
    for i in range(e_steps):
        for k, t in host.items():
            getattr(gd, k).copy_(t, non_blocking=True)
        rend.render(gd, [cams[args.warmup + i]], out=img, check=False)
        out_host[: 3 * RES * RES].copy_(img.rgb, non_blocking=True)
        out_host[3 * RES * RES: 6 * RES * RES].copy_(img.normal, non_blocking=True)
        out_host[6 * RES * RES:].copy_(img.depth, non_blocking=True)
    b.record(st)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / e_steps
    e2e_val = world * RES * RES / (e2e_ms / 1e3) / 1e6

    # roofline of the dominant stage
    peaks, src = measured_peaks()
    names = ["project", "sort_bin", "blend"]
    mean_stage = stage.mean(0)
    dom = int(np.argmax(mean_stage))
    K = rend.n_keys
    n = gs.n
    if dom == 0:
        alg = n * (48 + 44)
    elif dom == 1:
        alg = n * 16 + K * 12 + 6 * K * 24
    else:
        alg = K * (4 + 64) + RES * RES * 36
    achieved = alg / (mean_stage[dom] / 1e3) / 1e9
    roof = {"kernel": names[dom], "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
            "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": None,
            "peak_source": src}

    line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
            "p50_ms": float(np.percentile(frame_ms, 50)), "p99_ms": float(np.percentile(frame_ms, 99)),
            "stage_ms": {nm: float(x) for nm, x in zip(names, mean_stage)},
            "keys_per_frame": K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args.path), "points": N_POINTS, "resolution": RES,
                       "cameras": "uniform on a 2.5 m sphere, re-drawn per frame",
                       "l2": "flushed (256 MiB write) before every timed frame",
                       "tile": args.tile,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "clocks": clocks, "gpu_launches": 11 * args.steps,
            "e2e": {"value": e2e_val, "unit": "Mpix/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "roofline": roof}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

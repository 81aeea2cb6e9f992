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
            "pca": "800K-point humanoid proxy, 1 frame = kNN-PCA estimation of all points + "
                   "1024x1024 render (projection, binning, radix sort, compositing)",
            "learned": "800K-point humanoid proxy, 1 frame = kNN-PCA + learned MLP estimation of all "
                       "points + 1024x1024 render (projection, binning, radix sort, compositing)"}[path]


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


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value over all ranks (the slowest rank's time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, steps: int, pixels_per_step: int, max_ms: float) -> float:
    """Whole-job Mpix/s: the pixels every rank rendered over the slowest
    rank's time (each rank renders its own frames: replicas)."""
    return world * steps * pixels_per_step / (max_ms / 1e3) / 1e6


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def oracle_frame(xyz, rgb, g, cam, path):
    """One frame of the FP64 oracle: estimation (kNN-PCA) when the path has
    one, then projection, binning and compositing."""
    import oracle
    if path != "render":
        g = oracle.estimate_pca(xyz, rgb)
    p = oracle.project(g, cam)
    oracle.bin_keys([p], [cam])
    oracle.render(g, cam, proj=p)


def cpu_baseline(path: str, budget_s: float = 12.0) -> dict:
    """The FP64 oracle on the host cores, on a bounded sample of frames."""
    import oracle
    xyz, rgb, g = make_inputs()
    cams = cameras(xyz.mean(0), 64, SEED + 1)
    t0 = time.perf_counter()
    frames = 0
    while frames < len(cams) and (time.perf_counter() - t0) < budget_s:
        oracle_frame(xyz, rgb, g, cams[frames], path)
        frames += 1
    dt = time.perf_counter() - t0
    what = "kNN-PCA estimation + render" if path != "render" else "render"
    return {"value": frames * RES * RES / dt / 1e6, "unit": "Mpix/s", "cores": oracle.num_threads(),
            "kind": "oracle", "ms_per_frame": 1e3 * dt / frames,
            "sample": f"{frames} frames of the oracle's {what} of the 800K-point cloud at 1024x1024 "
                      f"(the oracle has no learned network; its frame is the kNN-PCA path)"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    t0 = time.perf_counter()
    import oracle
    xyz, rgb, g = make_inputs()
    cams = cameras(xyz.mean(0), args.warmup + args.steps, SEED + 1)
    times = []
    budget_s = 240.0  # the whole run stays within a few minutes: frames past it are not run
    for i, cam in enumerate(cams):
        t = time.perf_counter()
        oracle_frame(xyz, rgb, g, cam, "pca")
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
        if len(times) >= 3 and time.perf_counter() - t0 > budget_s:
            break
    tot = sum(times)
    val = len(times) * RES * RES / tot / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mpix/s", "n_gpus": world,
            "steps": len(times), "steps_requested": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / len(times),
            "p50_ms": 1e3 * float(np.percentile(times, 50)), "p99_ms": 1e3 * float(np.percentile(times, 99)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name("pca"), "points": N_POINTS,
                                            "resolution": RES},
            "cpu_baseline": {"value": val, "unit": "Mpix/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{len(times)} full frames (of {args.steps} requested; {budget_s:.0f} s "
                                       f"budget) after {args.warmup} warm-up"},
            "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default=None, choices=["render", "pca", "learned"])
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
    from paper_2409_16504_gb300.estimate import LEARNED, PCA, Estimator, cloud_tensors
    from paper_2409_16504_gb300.render import p2e_project, p2e_render, p2e_sort_bin

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    mlp_blob = learned_weights(dev)
    paths = [args.path] if args.path else (["learned", "pca"] if mlp_blob is not None else ["pca"])
    xyz, rgb, g = make_inputs()
    center = xyz.mean(0)
    e_steps = max(3, min(args.steps, 50))
    cams = cameras(center, args.warmup + max(args.steps, e_steps), SEED + 100 + rank)
    cx, cc = cloud_tensors(xyz, rgb, dev)
    g_static = GaussianSet.from_numpy(g, dev)
    est = Estimator(len(xyz), dev)
    gs = GaussianSet.empty(len(xyz), dev)
    st = torch.cuda.current_stream()
    rend = Renderer({"tile": args.tile}, capacity=1 << 21, device=dev)
    est(cx, cc, out=gs)
    rend.render(gs, [cams[0]])
    rend.capacity = int(rend.n_keys * 1.6) + 4096   # headroom for other viewpoints
    rend.render(gs, [cams[0]])
    img = Images([cams[0]], dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def frame(cam, path):
        es = [ev() for _ in range(5)]
        es[0].record(st)
        if path == "render":
            src = g_static
        else:
            est(cx, cc, mode=LEARNED if path == "learned" else PCA, mlp_blob=mlp_blob, out=gs)
            src = gs
        es[1].record(st)
        p2e_project(src, [cam], rend.cfg, rend.proj)
        es[2].record(st)
        p2e_sort_bin(rend.proj, src.n, [cam], rend.cfg, rend.bins)
        es[3].record(st)
        p2e_render(src, rend.proj, rend.bins, [cam], rend.cfg, img.rgb, img.normal, img.depth,
                   img.alpha, img.last)
        es[4].record(st)
        return es

    def timed(path):
        for i in range(args.warmup):
            flush.fill_(i & 0xFF)
            frame(cams[i], path)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        recs = []
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            recs.append(frame(cams[args.warmup + i], path))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        stage = np.array([[a.elapsed_time(b) for a, b in zip(r[:-1], r[1:])] for r in recs])
        return stage

    clk = Clocks(local)
    clk.start()
    results = {p: timed(p) for p in paths}
    clocks = clk.stop()
    st_ok, k = 0, rend.n_keys
    from paper_2409_16504_gb300 import p2e_bins_check
    st_ok, k = p2e_bins_check(rend.bins)
    if st_ok != 0:
        raise RuntimeError(f"binning status {st_ok}: key capacity {rend.capacity} < {k}")

    def summary(stage):
        fm = stage.sum(1)
        tot = max_over_ranks(float(fm.sum()), world, dev)
        return dict(value=job_throughput(world, args.steps, RES * RES, tot), ms=tot / args.steps,
                    p50=float(np.percentile(fm, 50)), p99=float(np.percentile(fm, 99)),
                    stage={nm: float(x) for nm, x in zip(["estimate", "project", "sort_bin", "blend"],
                                                         stage.mean(0))})
    sums = {p: summary(results[p]) for p in paths}
    head_path = paths[0]
    hs = sums[head_path]

    # end to end through the public API: every frame's cloud is uploaded
    # from pinned host memory and its rgb/normal/depth images are read back
    # to pinned host memory.  Uploads, compute (estimation + rendering) and
    # read-backs run on three streams, double-buffered, so that frame i+1's
    # upload and frame i-1's read-back overlap frame i's compute.
    hx, hc = cx.cpu().pin_memory(), cc.cpu().pin_memory()
    outs = [torch.empty((7 * RES * RES,), dtype=torch.float32).pin_memory() for _ in range(2)]
    dxs, dcs = [torch.empty_like(cx) for _ in range(2)], [torch.empty_like(cc) for _ in range(2)]
    imgs = [Images([cams[0]], dev) for _ in range(2)]
    h2d = (hx.numel() + hc.numel()) * 4
    d2h = outs[0].numel() * 4
    mode = LEARNED if head_path == "learned" else PCA
    cps, kst, dns = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    up_done = [torch.cuda.Event() for _ in range(2)]
    comp_done = [torch.cuda.Event() for _ in range(2)]
    down_done = [torch.cuda.Event() for _ in range(2)]
    torch.cuda.synchronize()
    for k in range(2):  # start from recorded events
        comp_done[k].record(kst)
        down_done[k].record(dns)

    def e2e_frame(i, cam):
        k = i & 1
        with torch.cuda.stream(cps):
            cps.wait_event(comp_done[k])            # frame i-2 done reading dxs[k]
            dxs[k].copy_(hx, non_blocking=True)
            dcs[k].copy_(hc, non_blocking=True)
            up_done[k].record(cps)
        with torch.cuda.stream(kst):
            kst.wait_event(up_done[k])
            kst.wait_event(down_done[k])            # frame i-2's images read back
            src = (est(dxs[k], dcs[k], mode=mode, mlp_blob=mlp_blob, out=gs, stream=kst)
                   if head_path != "render" else g_static)
            rend.render(src, [cam], out=imgs[k], check=False, stream=kst)
            comp_done[k].record(kst)
        with torch.cuda.stream(dns):
            dns.wait_event(comp_done[k])
            o = outs[k]
            o[: 3 * RES * RES].copy_(imgs[k].rgb, non_blocking=True)
            o[3 * RES * RES: 6 * RES * RES].copy_(imgs[k].normal, non_blocking=True)
            o[6 * RES * RES:].copy_(imgs[k].depth, non_blocking=True)
            down_done[k].record(dns)

    for w in range(4):
        e2e_frame(w, cams[w])
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record(cps)
    for i in range(e_steps):
        e2e_frame(i, cams[args.warmup + i])
    cps.wait_stream(dns)
    b.record(cps)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / e_steps

    # the rows beyond the frame: relighting of the 1024^2 view from its normal
    # image (HBM bound: 28 B read + 12 B written per pixel) and the global
    # isotropic estimator (kNN-PCA + mean spacing), each timed alone
    from paper_2409_16504_gb300 import relight
    lights = [(0.3, 0.8, -0.5, 0.9), (-1.0, 0.2, 0.1, 0.3)]
    shaded = torch.empty_like(img.rgb)

    def timed_op(fn, reps=20):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.fill_(1)
            x0, x1 = ev(), ev()
            x0.record(st)
            fn()
            x1.record(st)
            torch.cuda.synchronize()
            ts.append(x0.elapsed_time(x1))
        return float(np.median(ts))
    relight_ms = timed_op(lambda: relight(img, lights, ambient=0.15, out=shaded))
    relight_gbs = RES * RES * 40 / (relight_ms / 1e3) / 1e9
    glob_ms = timed_op(lambda: est.global_(cx, cc, 1.5, out=gs))
    from paper_2409_16504_gb300 import point_raster
    raster_img = Images([cams[0]], dev)
    raster_ms = timed_op(lambda: point_raster(cx, cc, [cams[0]], out=raster_img))

    # roofline of the dominant stage (one C-ABI call, timed by CUDA events on
    # its stream): algorithmic DRAM bytes per call / its mean duration
    peaks, src_peak = measured_peaks()
    dom = max(hs["stage"], key=hs["stage"].get)
    K, n = k, len(xyz)
    if dom == "blend":
        # per key: its index and the splat record gathered (xy_depth, conic,
        # rect, rgb, normal); per pixel the nine output planes
        alg = K * (4 + 16 + 16 + 8 + 16 + 16) + RES * RES * 36
        what = "p2e_render (compositing)"
    elif dom == "sort_bin":
        # depth keys of the Gaussians and four passes over them, emission of
        # the tile keys, two passes over those (12 B read + 12 B written each)
        alg = n * (4 + 16 + 12) + 4 * n * 24 + n * 16 + K * 12 + 2 * K * 24
        what = "p2e_sort_bin"
    elif dom == "project":
        alg = n * (48 + 44)
        what = "p2e_project"
    else:
        # kNN-PCA: points in (xyz, rgb), neighbour indices and Gaussians out;
        # the learned head then reads the indices, the neighbours' points and
        # the PCA Gaussians once and rewrites the Gaussians
        alg = n * (32 + 64 + 80)
        if head_path == "learned":
            alg += n * (64 + 32 + 80 + 64)
        what = "p2e_estimate (kNN-PCA" + (" + learned MLP)" if head_path == "learned" else ")")
    achieved = alg / (hs["stage"][dom] / 1e3) / 1e9
    roof = {"kernel": what, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": None,
            "peak_source": src_peak, "algorithmic_bytes_per_launch": alg}

    # launches per frame: estimate (init, bbox, grid, count, scan, scatter,
    # kNN-PCA [+ MLP]); project 1; sort_bin (scan+emit, histogram, radix
    # passes, ranges, work list); render (fill, item table, blend)
    passes = (32 + int(math.ceil(math.log2(max(2, (RES // args.tile) ** 2)))) + 7) // 8
    launches_sort = 4 + passes
    launches_per_frame = {"render": 1 + launches_sort + 3, "pca": 7 + 1 + launches_sort + 3,
                          "learned": 8 + 1 + launches_sort + 3}
    line = {"metric": METRIC, "value": hs["value"], "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": hs["ms"], "p50_ms": hs["p50"], "p99_ms": hs["p99"],
            "stage_ms": hs["stage"], "path": head_path,
            "paths": {p: {"Mpix_s": v["value"], "p50_ms": v["p50"], "p99_ms": v["p99"], "stage_ms": v["stage"]}
                      for p, v in sums.items()},
            "keys_per_frame": K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(head_path), "points": N_POINTS, "resolution": RES,
                       "cameras": "uniform on a 2.5 m sphere, re-drawn per frame",
                       "l2": "flushed (256 MiB write) before every timed frame", "tile": args.tile,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "clocks": clocks, "gpu_launches": sum(launches_per_frame[p] for p in paths) * args.steps,
            "e2e": {"value": world * RES * RES / (e2e_ms / 1e3) / 1e6, "unit": "Mpix/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "roofline": roof,
            "beyond_frame": {"relight_1024": {"ms": relight_ms, "achieved_gbs": relight_gbs,
                                              "frac_hbm": relight_gbs / peaks["hbm_gbs"]},
                             "global_estimate_800k_ms": glob_ms, "point_raster_800k_1024_ms": raster_ms}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(head_path)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def learned_weights(dev):
    """The trained estimator's weight blob, if the package ships one."""
    try:
        from paper_2409_16504_gb300 import mlp
    except ImportError:
        return None
    return mlp.load_trained(dev)


if __name__ == "__main__":
    main()

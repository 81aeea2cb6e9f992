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
stream, and the dominant kernels inside it with CUDA events that the
library records around their launches (p2e_set_kernel_probe).

Besides the timed steps the line carries: the per-frame latency
distribution over 1000 frames per path; the end-to-end latency of single
frames through the public API (upload of the cloud from pinned memory,
estimation, rendering, read-back of the images); the overlapped end-to-end
throughput; a short serving run (Poisson viewpoint requests at 500/s
against a moving cloud); and the rooflines of the kNN, compositing and MLP
kernels.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import ctypes as C
import hashlib
import json
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
LATENCY_FRAMES = 1000
E2E_LATENCY_FRAMES = 200

# Algorithmic work per unit (the roofline numerators).
#   kNN: per query ~27 grid cells x ~3 points x 16 B (a float4 per candidate)
KNN_BYTES_PER_QUERY = 27 * 3 * 16
#   MLP head: 2 (96*64 + 64*64*2 + 64*8) flop per point
MLP_FLOP_PER_POINT = 2 * (96 * 64 + 64 * 64 * 2 + 64 * 8)
#   compositing: per evaluated (pixel, splat) pair ~20 fp32 operations (the
#   pixel offset 4, the conic form 8, exp + alpha 3, transmittance 2, the
#   seven weighted sums and the weight 8 for a contributing splat) and one
#   ex2 on the MUFU pipe; HBM: per key its index and gathered record
#   (xy_depth, conic, rect, rgb, normal: 4 + 16 + 16 + 8 + 16 + 16 B) and
#   per pixel the nine output planes
BLEND_FP32_PER_PAIR = 20
BLEND_BYTES_PER_KEY = 4 + 16 + 16 + 8 + 16 + 16
BLEND_BYTES_PER_PIXEL = 9 * 4
#   projection (one kernel): per Gaussian 48 B read (mean_op, scale, quat) and
#   44 B written (xy_depth, conic_op, rect, tile count)
PROJECT_BYTES_PER_GAUSSIAN = 48 + 44
#   binning (a stage of ~12 launches, depth-first order): per Gaussian the
#   depth key built (8 B read + 12 B written), four 8-bit passes over the
#   depth keys (12 B read + 12 B written each) and the emission's read of its
#   record and sorted index (24 B); per tile key its emission (12 B), two passes
#   over the tile bits (24 B each) and the range search (8 B)
SORT_BYTES_PER_GAUSSIAN = 20 + 4 * 24 + 24
SORT_BYTES_PER_KEY = 12 + 2 * 24 + 8
FP32_LANES_PER_SM = 128
#   backward compositing (the per-tile kernel of the differentiation), counted
#   like the forward: per evaluated (pixel, splat) pair the offset and conic
#   form in each of its two walks (2 x 12); per contributing pair exp +
#   alpha and the transmittance in the front-to-back walk (5), and in the
#   back-to-front walk exp + alpha (3), 1 - alpha, T_k, the weight, the
#   seven-channel upstream dot (7), dL/dalpha (3), the running tail, the
#   seven weighted channels (7) and the geometric gradients o, A, B, C, u, v
#   (16): 37 (the per-splat reduction over the warp is counted as data
#   movement, not arithmetic; the warp reductions are reported beside).
#   HBM: per key its index and record in both walks
#   (4 + 16 + 16 + 8, then 4 + 16 + 16 + 8 + 16 + 16 B), per pixel the
#   upstream rgb and normal planes and `last` (28 B), per (view, Gaussian)
#   its 13-float gradient slot (52 B)
BWD_FP32_PER_EVAL = 2 * (4 + 8)
BWD_FP32_PER_CONTRIB = 5 + 3 + 37
BWD_BYTES_PER_KEY = (4 + 16 + 16 + 8) + (4 + 16 + 16 + 8 + 16 + 16)
BWD_BYTES_PER_PIXEL = 12 + 12 + 4
BWD_BYTES_PER_SLOT = 13 * 4

# DRAM bytes per launch from one ncu capture of the kernel (dram__bytes_read
# + dram__bytes_write, profiles/), valid while the kernel's sources are
# unchanged (the SHA-256 prefix of their concatenation below); otherwise the
# line reports null.
_CSRC = "paper_2409_16504_gb300/csrc/"
NCU_TRAFFIC = {
    # the kNN search's two launches per frame (counting, selection), summed
    "knn": {"kernel": "knn_count_kernel + knn_select_kernel", "sources": [_CSRC + "estimate.cu"],
            "sha256_16": "c39e882389eab2c2", "bytes": 32_422_000},
    "blend": {"kernel": "blend_kernel<8>", "tile": 8, "sources": [_CSRC + "blend.cu", _CSRC + "splat.cuh"],
              "sha256_16": "ae1d3d0a5411ef65", "bytes": 373_008_000},
    "mlp": {"kernel": "mlp_estimate_kernel", "sources": [_CSRC + "mlp.cu", _CSRC + "tcgen05.cuh"],
            "sha256_16": "7d49e064b1b85464", "bytes": 135_280_000},
    "project": {"kernel": "project_kernel", "sources": [_CSRC + "project.cu"],
                "sha256_16": "aff9ed682ee64b66", "bytes": 40_470_000},
    # the whole binning stage of one learned frame (12 launches: depth keys,
    # six radix passes, emission, ranges, work list), the mean of the steady
    # frames of one capture (~3.0M keys)
    "sort_bin": {"kernel": "p2e_sort_bin stage", "tile": 8, "sources": [_CSRC + "sort.cu"],
                 "sha256_16": "df8143ffee336acc", "bytes": 218_800_000},
    # the backward's compositing part (walk ends, item table, folds, gradient
    # walks), one launch each, on the differentiation workload
    "blend_bwd": {"kernel": "bwd_tile_end + bwd_items + bwd_fold + blend_bwd_kernel<8>", "tile": 8,
                  "sources": [_CSRC + "backward.cu", _CSRC + "splat.cuh"],
                  "sha256_16": "0c583b337e23d57c", "bytes": 313_622_528},
}


def source_digest(rels: list) -> str:
    h = hashlib.sha256()
    for rel in rels:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(which: str, tile: int | None = None):
    """The captured DRAM bytes per launch, or None when the sources changed
    since the capture or (for a tile-templated kernel) the tile differs."""
    e = NCU_TRAFFIC[which]
    if e["bytes"] is None or e["sha256_16"] != source_digest(e["sources"]):
        return None
    if tile is not None and e.get("tile", tile) != tile:
        return None
    return e["bytes"]


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
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def pct(a, q):
    return float(np.percentile(np.asarray(a), q)) if len(a) else None


WEIGHTS = os.path.join(ROOT, "paper_2409_16504_gb300", "weights", "estimator.npz")


def oracle_params():
    """The shipped network weights as plain arrays (the data both arms use)."""
    z = np.load(WEIGHTS)
    return {k: z[k] for k in z.files}


def oracle_frame(xyz, rgb, g, cam, path, params=None):
    """One frame of the FP64 oracle: estimation (kNN-PCA, and for the
    learned path the network's corrections with the forward's bf16
    roundings) when the path has one, then projection, binning and
    compositing."""
    import oracle
    if path == "learned":
        from oracle import mlp as om
        e = om.estimate(xyz, rgb, params if params is not None else oracle_params())
        f32 = lambda a: np.asarray(a, np.float32)  # noqa: E731
        g = dict(mean=f32(xyz), scale=f32(e["scale"]), quat=f32(e["quat"]), opacity=f32(e["opacity"]),
                 rgb=f32(rgb), normal=f32(e["normal"]))
    elif path != "render":
        g = oracle.estimate_pca(xyz, rgb)
    p = oracle.project(g, cam)
    oracle.bin_keys([p], [cam])
    oracle.render(g, cam, proj=p)


def cpu_baseline(path: str, budget_s: float = 12.0) -> dict:
    """The FP64 oracle on the host cores, on a bounded sample of frames."""
    import oracle
    xyz, rgb, g = make_inputs()
    cams = cameras(xyz.mean(0), 64, SEED + 1)
    params = oracle_params() if path == "learned" else None
    t0 = time.perf_counter()
    frames = 0
    while frames < len(cams) and (time.perf_counter() - t0) < budget_s:
        oracle_frame(xyz, rgb, g, cams[frames], path, params)
        frames += 1
    dt = time.perf_counter() - t0
    what = {"learned": "kNN-PCA + learned-network estimation + render", "pca": "kNN-PCA estimation + render",
            "render": "render"}[path]
    return {"value": frames * RES * RES / dt / 1e6, "unit": "Mpix/s", "cores": oracle.num_threads(),
            "kind": "oracle", "ms_per_frame": 1e3 * dt / frames,
            "sample": f"{frames} frames of the oracle's {what} of the 800K-point cloud at 1024x1024"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    t0 = time.perf_counter()
    import oracle
    xyz, rgb, g = make_inputs()
    cams = cameras(xyz.mean(0), args.warmup + args.steps, SEED + 1)
    path = args.path or "learned"  # the workload our arm's line is quoted on
    params = oracle_params() if path == "learned" else None
    times = []
    budget_s = 240.0  # the whole run stays within a few minutes: frames past it are not run
    for i, cam in enumerate(cams):
        t = time.perf_counter()
        oracle_frame(xyz, rgb, g, cam, path, params)
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
            "data": "synthetic", "config": {"workload": workload_name(path), "points": N_POINTS,
                                            "resolution": RES},
            "cpu_baseline": {"value": val, "unit": "Mpix/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{len(times)} full frames (of {args.steps} requested; {budget_s:.0f} s "
                                       f"budget) after {args.warmup} warm-up"},
            "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


class Probe:
    """CUDA events (and an optional device counter) that libp2e records
    around one kernel's launches, one event pair per step."""

    def __init__(self, kernel: int, steps: int, dev, counters: int = 0):
        import torch
        from paper_2409_16504_gb300 import _lib
        self.lib, self.kernel = _lib.load(), kernel
        self.ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(steps)]
        for a, b in self.ev:   # create the underlying events
            a.record()
            b.record()
        torch.cuda.synchronize()
        self.count = torch.zeros(counters, dtype=torch.int64, device=dev) if counters else None
        self.armed = []

    def arm(self, i: int):
        from paper_2409_16504_gb300 import _lib
        a, b = self.ev[i]
        p = _lib.P2EKernelProbe(a.cuda_event, b.cuda_event,
                                self.count.data_ptr() if self.count is not None else None)
        _lib.check("p2e_set_kernel_probe", self.lib.p2e_set_kernel_probe(self.kernel, C.byref(p)))
        self.armed.append(i)

    def disarm(self):
        self.lib.p2e_set_kernel_probe(self.kernel, None)

    def mean_ms(self) -> float:
        return float(np.mean([self.ev[i][0].elapsed_time(self.ev[i][1]) for i in self.armed]))

    def per_step_count(self, i: int = 0) -> float:
        return float(self.count[i].item()) / max(len(self.armed), 1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--path", default=None, choices=["render", "pca", "learned"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the timed steps (for profiler runs): no latency, end-to-end or serving runs")
    ap.add_argument("--tile", type=int, default=8, choices=[8, 16, 32],
                    help="binning tile in pixels (8: measured fastest for the 1024^2 frames)")
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

    from paper_2409_16504_gb300 import GaussianSet, Images, Renderer, _lib, p2e_bins_check
    from paper_2409_16504_gb300.estimate import LEARNED, PCA, Estimator, cloud_tensors
    from paper_2409_16504_gb300.render import p2e_project, p2e_render, p2e_sort_bin

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    mlp_blob = learned_weights(dev)
    paths = [args.path] if args.path else (["learned", "pca"] if mlp_blob is not None else ["pca"])
    xyz, rgb, g = make_inputs()
    n = len(xyz)
    center = xyz.mean(0)
    n_lat = 0 if args.no_extras else LATENCY_FRAMES
    cams = cameras(center, args.warmup + max(args.steps, n_lat, E2E_LATENCY_FRAMES), SEED + 100 + rank)
    cx, cc = cloud_tensors(xyz, rgb, dev)
    g_static = GaussianSet.from_numpy(g, dev)
    est = Estimator(n, dev)
    gs = GaussianSet.empty(n, dev)
    st = torch.cuda.current_stream()
    rend = Renderer({"tile": args.tile}, capacity=1 << 21, device=dev)
    # key buffers: twice the first view's keys under the estimate that needs
    # the most (headroom for other viewpoints and the compositing states)
    first = 0
    for m in ([PCA, LEARNED] if mlp_blob is not None else [PCA]):
        est(cx, cc, mode=m, mlp_blob=mlp_blob, out=gs)
        rend.render(gs, [cams[0]])
        first = max(first, rend.n_keys)
    rend.capacity = int(first * 2.0) + 4096
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
        """The K timed steps, with the kernel probes armed on every step."""
        probes = {"knn": Probe(_lib.P2E_PROBE_KNN, args.steps, dev) if path != "render" else None,
                  "mlp": Probe(_lib.P2E_PROBE_MLP, args.steps, dev) if path == "learned" else None,
                  "blend": Probe(_lib.P2E_PROBE_BLEND, args.steps, dev, counters=1)}
        for i in range(args.warmup):
            flush.fill_(i & 0xFF)
            frame(cams[i], path)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        recs = []
        keys = torch.zeros((), dtype=torch.int64, device=dev)  # summed key counts (device side)
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            for p in probes.values():
                if p is not None:
                    p.arm(i)
            recs.append(frame(cams[args.warmup + i], path))
            keys += rend.bins.counters[0]  # after the frame's last event: outside its timing
        for p in probes.values():
            if p is not None:
                p.disarm()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        stage = np.array([[a.elapsed_time(b) for a, b in zip(r[:-1], r[1:])] for r in recs])
        kern = {k: (p.mean_ms() if p is not None else None) for k, p in probes.items()}
        pairs = probes["blend"].per_step_count()
        return stage, kern, pairs, float(keys.item()) / args.steps

    def latency(path, frames):
        """Per-frame device latency (estimate + project + sort + blend) over
        `frames` frames, L2 flushed before each, cameras re-drawn."""
        for i in range(3):
            frame(cams[i], path)
        out = []
        for i in range(frames):
            flush.fill_(i & 0xFF)
            es = frame(cams[i], path)
            out.append(es)
            if (i + 1) % 64 == 0:   # bound the work in flight; the host stays frames ahead
                torch.cuda.synchronize()
        torch.cuda.synchronize()
        return np.array([e[0].elapsed_time(e[-1]) for e in out])

    clk = Clocks(local)
    clk.start()
    results = {p: timed(p) for p in paths}
    clocks = clk.stop()
    st_ok, last_keys = p2e_bins_check(rend.bins)
    if st_ok != 0:
        raise RuntimeError(f"binning / compositing status {st_ok} (key capacity {rend.capacity}, {last_keys} keys)")

    def summary(stage):
        fm = stage.sum(1)
        tot = max_over_ranks(float(fm.sum()), world, dev)
        return dict(value=job_throughput(world, args.steps, RES * RES, tot), ms=tot / args.steps,
                    p50=float(np.percentile(fm, 50)), p99=float(np.percentile(fm, 99)),
                    stage={nm: float(x) for nm, x in zip(["estimate", "project", "sort_bin", "blend"],
                                                         stage.mean(0))})
    sums = {p: summary(results[p][0]) for p in paths}
    head_path = paths[0]
    hs = sums[head_path]
    kern, pairs, n_keys = results[head_path][1], results[head_path][2], results[head_path][3]
    assert n_keys > n // 2, n_keys  # mean keys per timed frame of the reported path
    lat = {p: latency(p, n_lat) for p in paths} if n_lat else {}

    # ---- kernel rooflines (achieved work per launch / CUDA-event duration)
    peaks, src_peak = measured_peaks()
    hbm = peaks["hbm_gbs"]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = sms * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12   # TFLOP/s (one op per lane per clock)
    rooflines = {}
    if kern["knn"]:
        alg = KNN_BYTES_PER_QUERY * n
        a = alg / (kern["knn"] / 1e3) / 1e9
        rooflines["knn"] = {"kernel": "knn_count_kernel + knn_select_kernel", "bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s",
                            "frac": a / hbm, "traffic": ncu_traffic("knn"), "ms": kern["knn"],
                            "algorithmic_bytes_per_launch": alg, "peak_source": src_peak}
    if kern["mlp"]:
        alg = MLP_FLOP_PER_POINT * n
        a = alg / (kern["mlp"] / 1e3) / 1e12
        pk = peaks["bf16_tflops"]
        rooflines["mlp"] = {"kernel": "mlp_estimate_kernel", "bound": "tensor", "achieved": a, "peak": pk,
                            "unit": "TFLOP/s", "frac": a / pk, "traffic": ncu_traffic("mlp"), "ms": kern["mlp"],
                            "algorithmic_flop_per_launch": alg, "peak_source": src_peak + " (bf16 burst)"}
    if kern["blend"]:
        a = BLEND_FP32_PER_PAIR * pairs / (kern["blend"] / 1e3) / 1e12
        hb = (BLEND_BYTES_PER_KEY * n_keys + BLEND_BYTES_PER_PIXEL * RES * RES) / (kern["blend"] / 1e3) / 1e9
        rooflines["blend"] = {"kernel": f"blend_kernel<{args.tile}>", "bound": "alu", "achieved": a,
                              "peak": fp32_peak, "unit": "TFLOP/s", "frac": a / fp32_peak,
                              "traffic": ncu_traffic("blend", args.tile), "ms": kern["blend"],
                              "pairs_per_launch": pairs, "fp32_ops_per_pair": BLEND_FP32_PER_PAIR,
                              "peak_derivation": f"{sms} SMs x {FP32_LANES_PER_SM} fp32 lanes x {sm_mhz:.0f} MHz",
                              "hbm": {"achieved_gbs": hb, "frac": hb / hbm,
                                      "algorithmic_bytes_per_launch": BLEND_BYTES_PER_KEY * n_keys +
                                      BLEND_BYTES_PER_PIXEL * RES * RES}}
    # stage rooflines from the stage events (projection is one launch; binning
    # is a stage of several, reported as such)
    a = PROJECT_BYTES_PER_GAUSSIAN * n / (hs["stage"]["project"] / 1e3) / 1e9
    rooflines["project"] = {"kernel": "project_kernel", "bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s",
                            "frac": a / hbm, "traffic": ncu_traffic("project"), "ms": hs["stage"]["project"],
                            "algorithmic_bytes_per_launch": PROJECT_BYTES_PER_GAUSSIAN * n,
                            "peak_source": src_peak, "timed": "stage events (one launch)"}
    alg = SORT_BYTES_PER_GAUSSIAN * n + SORT_BYTES_PER_KEY * n_keys
    a = alg / (hs["stage"]["sort_bin"] / 1e3) / 1e9
    rooflines["sort_bin"] = {"kernel": "p2e_sort_bin stage (depth keys, 6 radix passes, emission, ranges)",
                             "bound": "hbm", "achieved": a, "peak": hbm, "unit": "GB/s", "frac": a / hbm,
                             "traffic": ncu_traffic("sort_bin", args.tile), "ms": hs["stage"]["sort_bin"],
                             "algorithmic_bytes_per_call": alg,
                             "peak_source": src_peak, "timed": "stage events (~12 launches)"}
    dom = max((k for k in rooflines if k != "sort_bin"), key=lambda k: rooflines[k]["ms"])  # one kernel

    line = {"metric": METRIC, "value": hs["value"], "unit": "Mpix/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": hs["ms"], "p50_ms": hs["p50"], "p99_ms": hs["p99"],
            "stage_ms": hs["stage"], "kernel_ms": kern, "path": head_path,
            "paths": {p: {"Mpix_s": v["value"], "p50_ms": v["p50"], "p99_ms": v["p99"], "stage_ms": v["stage"],
                          "kernel_ms": results[p][1], "keys_per_frame": results[p][3]} for p, v in sums.items()},
            "keys_per_frame": n_keys, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(head_path), "points": N_POINTS, "resolution": RES,
                       "cameras": "uniform on a 2.5 m sphere, re-drawn per frame",
                       "l2": "flushed (256 MiB write) before every timed frame", "tile": args.tile,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "clocks": clocks, "roofline": rooflines[dom], "rooflines": rooflines}
    if lat:
        line["latency"] = {p: {"frames": len(v), "p50_ms": pct(v, 50), "p99_ms": pct(v, 99),
                               "max_ms": float(v.max()), "under_10ms": float((v < 10.0).mean())}
                           for p, v in lat.items()}

    # launches of our kernels per frame: estimate (init, bbox, grid, count,
    # scan, scatter, kNN-PCA, listed queries [+ MLP head]); project; sort_bin
    # (depth min, depth keys, 4 depth passes, scan + emit, digit histogram,
    # tile passes, ranges, work list); render (fill, item table, blend)
    tbits = int(np.ceil(np.log2(max(2, (RES // args.tile) ** 2))))
    tile_passes = (32 + tbits + 7) // 8 - 4
    sort_launches = 2 + 4 + 1 + 1 + tile_passes + 2
    per_frame = {"render": 1 + sort_launches + 3, "pca": 8 + 1 + sort_launches + 3,
                 "learned": 9 + 1 + sort_launches + 3}
    line["gpu_launches"] = sum(per_frame[p] for p in paths) * args.steps

    if not args.no_extras:
        line["e2e"] = e2e_runs(torch, dev, head_path, est, rend, mlp_blob, cx, cc, g_static, gs, cams, args, world)
        line["beyond_frame"] = beyond_frame(torch, dev, est, cx, cc, gs, img, cams, flush, ev, st, hbm)
        # differentiation at scale: 200K points, 8 views at 512^2, Eq. 5 + SSIM
        from paper_2409_16504_gb300.train import time_differentiation
        bp = Probe(_lib.P2E_PROBE_BLEND_BWD, 5, dev, counters=3)
        df = time_differentiation(points=200_000, views=8, res=512, ssim_weight=0.2, reps=5, probe=bp)
        ms = bp.mean_ms()
        n_eval, n_contrib, n_red = (bp.per_step_count(i) for i in range(3))
        ops = BWD_FP32_PER_EVAL * n_eval + BWD_FP32_PER_CONTRIB * n_contrib
        a = ops / (ms / 1e3) / 1e12
        hb = BWD_BYTES_PER_KEY * df["keys"] + BWD_BYTES_PER_PIXEL * df["pixels"] + \
            BWD_BYTES_PER_SLOT * df["points"] * df["views"]
        line["rooflines"]["blend_bwd"] = {
            "kernel": f"bwd_items + bwd_fold + blend_bwd_kernel<{df['tile']}> (the backward's compositing)",
            "bound": "alu", "achieved": a, "peak": fp32_peak,
            "unit": "TFLOP/s", "frac": a / fp32_peak, "traffic": ncu_traffic("blend_bwd", df["tile"]), "ms": ms,
            "workload": f"differentiation: {df['points']} points x {df['views']} views at {df['res']}^2",
            "pairs_evaluated_per_launch": n_eval, "pairs_contributing_per_launch": n_contrib,
            "warp_reductions_per_launch": n_red, "fp32_ops_per_launch": ops,
            "peak_derivation": f"{sms} SMs x {FP32_LANES_PER_SM} fp32 lanes x {sm_mhz:.0f} MHz",
            "hbm": {"achieved_gbs": hb / (ms / 1e3) / 1e9, "frac": hb / (ms / 1e3) / 1e9 / hbm,
                    "algorithmic_bytes_per_launch": hb}}
        line["differentiation"] = df
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(head_path)
    if rank == 0 and world == 1 and not args.no_serving and not args.no_extras:
        from paper_2409_16504_gb300 import serve
        torch.cuda.synchronize()
        line["serving"] = serve.run_load(seconds=3.0, rate=500.0, learned=mlp_blob is not None)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def e2e_runs(torch, dev, head_path, est, rend, mlp_blob, cx, cc, g_static, gs, cams, args, world):
    """End to end through the public API.  Every frame uploads its cloud
    from pinned host memory and reads its rgb/normal/depth images back to
    pinned host memory.
      * throughput: uploads, compute (estimation + rendering) and read-backs
        on three streams, double-buffered, so that frame i+1's upload and
        frame i-1's read-back overlap frame i's compute;
      * latency: single frames, one at a time: host clock from issuing the
        upload to observing the read-back complete."""
    from paper_2409_16504_gb300 import Images
    from paper_2409_16504_gb300.estimate import LEARNED, PCA
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    e_steps = max(3, min(args.steps, 50))
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
    for j in range(2):  # start from recorded events
        comp_done[j].record(kst)
        down_done[j].record(dns)

    def e2e_frame(i, cam):
        j = i & 1
        with torch.cuda.stream(cps):
            cps.wait_event(comp_done[j])            # frame i-2 done reading dxs[j]
            dxs[j].copy_(hx, non_blocking=True)
            dcs[j].copy_(hc, non_blocking=True)
            up_done[j].record(cps)
        with torch.cuda.stream(kst):
            kst.wait_event(up_done[j])
            kst.wait_event(down_done[j])            # frame i-2's images read back
            src = (est(dxs[j], dcs[j], mode=mode, mlp_blob=mlp_blob, out=gs, stream=kst)
                   if head_path != "render" else g_static)
            rend.render(src, [cam], out=imgs[j], check=False, stream=kst)
            comp_done[j].record(kst)
        with torch.cuda.stream(dns):
            dns.wait_event(comp_done[j])
            o = outs[j]
            o[: 3 * RES * RES].copy_(imgs[j].rgb, non_blocking=True)
            o[3 * RES * RES: 6 * RES * RES].copy_(imgs[j].normal, non_blocking=True)
            o[6 * RES * RES:].copy_(imgs[j].depth, non_blocking=True)
            down_done[j].record(dns)

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

    # single frames, one at a time, on one stream
    lat_host, lat_dev = [], []
    s = kst
    for i in range(3 + E2E_LATENCY_FRAMES):
        cam = cams[i]
        x0, x1 = ev(), ev()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with torch.cuda.stream(s):
            x0.record(s)
            dxs[0].copy_(hx, non_blocking=True)
            dcs[0].copy_(hc, non_blocking=True)
            src = (est(dxs[0], dcs[0], mode=mode, mlp_blob=mlp_blob, out=gs, stream=s)
                   if head_path != "render" else g_static)
            rend.render(src, [cam], out=imgs[0], check=False, stream=s)
            o = outs[0]
            o[: 3 * RES * RES].copy_(imgs[0].rgb, non_blocking=True)
            o[3 * RES * RES: 6 * RES * RES].copy_(imgs[0].normal, non_blocking=True)
            o[6 * RES * RES:].copy_(imgs[0].depth, non_blocking=True)
            x1.record(s)
        x1.synchronize()
        t1 = time.perf_counter()
        if i >= 3:
            lat_host.append(1e3 * (t1 - t0))
            lat_dev.append(x0.elapsed_time(x1))
    return {"value": world * RES * RES / (e2e_ms / 1e3) / 1e6, "unit": "Mpix/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
            "overlap": "uploads, compute and read-backs on three streams, double-buffered",
            "frame_latency": {"frames": len(lat_host), "p50_ms": pct(lat_host, 50), "p99_ms": pct(lat_host, 99),
                              "max_ms": float(max(lat_host)), "device_p50_ms": pct(lat_dev, 50),
                              "device_p99_ms": pct(lat_dev, 99),
                              "what": "one frame at a time: host clock from issuing the H2D upload of the "
                                      "cloud to the D2H read-back of rgb/normal/depth observed complete"}}


def beyond_frame(torch, dev, est, cx, cc, gs, img, cams, flush, ev, st, hbm):
    """The rows beyond the frame, each timed alone: relighting of the
    1024^2 view from its normal image (28 B read + 12 B written per pixel),
    the global isotropic estimator, the point raster."""
    from paper_2409_16504_gb300 import Images, point_raster, relight
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
    raster_img = Images([cams[0]], dev)
    raster_ms = timed_op(lambda: point_raster(cx, cc, [cams[0]], out=raster_img))
    return {"relight_1024": {"ms": relight_ms, "achieved_gbs": relight_gbs, "frac_hbm": relight_gbs / hbm},
            "global_estimate_800k_ms": glob_ms, "point_raster_800k_1024_ms": raster_ms}


def learned_weights(dev):
    """The trained estimator's weight blob, if the package ships one."""
    try:
        from paper_2409_16504_gb300 import mlp
    except ImportError:
        return None
    return mlp.load_trained(dev)


if __name__ == "__main__":
    main()

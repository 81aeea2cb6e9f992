"""Continuous-batching viewpoint server for a dynamic point cloud.

The paper's application streams a point-cloud video and renders every
incoming viewpoint within the 10 ms motion-to-photon budget, with
preprocessing (estimation) pipelined against rendering (Sec. 4.2, on two
GPUs there).  On one GB300 the two run on separate CUDA streams:

* cloud frames arrive at their own rate; each is estimated on the
  estimation stream into the back buffer of a double-buffered, resident
  Gaussian set and becomes the front buffer once its event completes;
* viewpoint requests (mixed resolutions) queue up; the scheduler admits
  them in arrival order into a batch while a slot is free and the batch's
  device memory fits the budget, and launches the batch as ONE multi-view
  project / sort / render call on the slot's stream against the current
  front buffer.  Requests that arrive while earlier batches are on the GPU
  go into the next batch on another slot, so batches overlap on the device;
* a request completes when its batch's event does; its latency is arrival
  to observed completion, on the host clock.

Each view's arithmetic does not depend on the other views of its batch
(tile ids are offset per view, a tile's list holds only its view's
splats), so a request's image is bit-identical alone and in any mix.

:class:`Scheduler` is the host-side policy, :class:`GpuExecutor` the device
side; tests drive the scheduler with a fake executor and a fake clock.
"""
from __future__ import annotations

import argparse
import math
import os
import sys
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

BYTES_PER_PIXEL = 9 * 4        # rgb 3, normal 3, depth, alpha, last
KEY_BYTES = 2 * (8 + 4)        # double-buffered key + value


@dataclass
class Request:
    rid: int
    camera: dict
    arrival: float
    admitted: float | None = None
    done: float | None = None
    batch: int | None = None
    images: dict | None = None
    dropped: bool = False

    @property
    def pixels(self) -> int:
        return int(self.camera["width"]) * int(self.camera["height"])

    @property
    def latency(self) -> float | None:
        return None if self.done is None else self.done - self.arrival


@dataclass
class Batch:
    bid: int
    requests: list
    slot: int
    mem: int
    handle: object = None
    launched: float = 0.0


@dataclass
class Scheduler:
    """Admission and batching policy (host only).

    ``mem_budget``: device bytes that in-flight batches may hold; a request
    costs its image planes plus ``keys_per_pixel`` key slots per pixel.
    ``slots``: batches in flight at once.  ``max_views``: views per batch.
    ``deadline``: if set, a request still pending that long after its
    arrival is dropped (completed unrendered, ``dropped`` set): a view
    shown after the motion-to-photon budget is of no use to the viewer.
    """
    executor: object
    slots: int = 3
    max_views: int = 8
    mem_budget: int = 4 << 30
    keys_per_pixel: float = 1.5
    deadline: float | None = None
    clock: object = time.perf_counter
    pending: deque = field(default_factory=deque)
    inflight: list = field(default_factory=list)
    finished: list = field(default_factory=list)
    next_rid: int = 0
    next_bid: int = 0

    def cost(self, req: Request) -> int:
        return int(req.pixels * (BYTES_PER_PIXEL + self.keys_per_pixel * KEY_BYTES))

    def submit(self, camera: dict, arrival: float | None = None) -> Request:
        r = Request(self.next_rid, camera, self.clock() if arrival is None else arrival)
        self.next_rid += 1
        if self.cost(r) > self.mem_budget:
            raise ValueError(f"request {r.rid} needs {self.cost(r)} B, more than the budget")
        self.pending.append(r)
        return r

    def mem_in_use(self) -> int:
        return sum(b.mem for b in self.inflight)

    def poll(self) -> list:
        """Completes every in-flight batch whose device work has finished."""
        done_now = []
        for b in list(self.inflight):
            if self.executor.query(b.handle):
                t = self.clock()
                for r in b.requests:
                    r.done = t
                    r.images = self.executor.result(b.handle, r)
                self.inflight.remove(b)
                self.executor.release(b.handle)
                self.finished.extend(b.requests)
                done_now.extend(b.requests)
        return done_now

    def admit(self) -> Batch | None:
        """Forms and launches one batch if a slot is free and the oldest
        pending request fits the memory left; later requests join while
        they fit (arrival order is kept)."""
        if self.deadline is not None:
            t = self.clock()
            while self.pending and t - self.pending[0].arrival > self.deadline:
                r = self.pending.popleft()
                r.done, r.dropped = t, True
                self.finished.append(r)
        if not self.pending or len(self.inflight) >= self.slots:
            return None
        free = self.mem_budget - self.mem_in_use()
        take, mem = [], 0
        while self.pending and len(take) < self.max_views:
            c = self.cost(self.pending[0])
            if mem + c > free:
                break
            mem += c
            take.append(self.pending.popleft())
        if not take:
            return None
        used = {b.slot for b in self.inflight}
        slot = next(s for s in range(self.slots) if s not in used)
        t = self.clock()
        b = Batch(self.next_bid, take, slot, mem, launched=t)
        self.next_bid += 1
        for r in take:
            r.admitted, r.batch = t, b.bid
        b.handle = self.executor.launch(slot, [r.camera for r in take])
        self.inflight.append(b)
        return b

    def step(self) -> None:
        self.poll()
        while self.admit() is not None:
            pass

    def drain(self, timeout: float = 30.0) -> None:
        t0 = time.perf_counter()
        while (self.pending or self.inflight) and time.perf_counter() - t0 < timeout:
            self.step()
            time.sleep(0.0001)


class GpuExecutor:
    """Device side: resident double-buffered Gaussians estimated per cloud
    frame on an estimation stream; one render slot (stream + buffers) per
    in-flight batch.

    A newly estimated buffer becomes the front buffer only once its
    estimation event has completed, so a batch never waits for estimation;
    the back buffer is rewritten only after every batch that read it has
    finished (the estimation stream waits on their events).
    """

    def __init__(self, n_max: int, slots: int, mlp_blob=None, cfg: dict | None = None, device="cuda",
                 keep_images: bool = False, capacity: int = 1 << 22):
        import torch
        from .estimate import LEARNED, PCA, Estimator
        from .render import GaussianSet, Renderer
        self.torch = torch
        self.device = device
        self.mode = LEARNED if mlp_blob is not None else PCA
        self.blob = mlp_blob
        self.est = Estimator(n_max, device)
        self.est_stream = torch.cuda.Stream(device=device)
        self.buffers = [GaussianSet.empty(n_max, device) for _ in range(2)]
        self.stage_xyz = torch.empty((n_max, 4), dtype=torch.float32, device=device)
        self.stage_rgb = torch.empty((n_max, 4), dtype=torch.float32, device=device)
        self.n = [0, 0]
        self.ready = [None, None]           # event: estimate of the buffer finished
        self.last_use = [[], []]            # events of batches that read the buffer
        self.front = None
        self.pending = None                 # buffer being estimated, not yet front
        self.version = [-1, -1]             # cloud frame held by each buffer
        self.streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self.renderers = [Renderer(cfg, capacity=capacity, device=device) for _ in range(slots)]
        self.keep_images = keep_images
        self.rerenders = 0

    def _promote(self) -> None:
        if self.pending is not None and self.ready[self.pending].query():
            # the estimate finished: raises if one of its bounded device
            # waits gave up (its Gaussians would be invalid)
            self.est.check(self.n[self.pending], self.est_stream)
            self.front, self.pending = self.pending, None

    def publish(self, xyz, rgb, version: int = 0) -> None:
        """Estimates a new cloud frame into the back buffer (asynchronous).

        ``xyz``/``rgb`` are (n, 4) float32 tensors; host tensors (pinned,
        unchanged until the estimate completes) are copied to the device on
        the estimation stream first."""
        torch = self.torch
        back = 1 if self.front == 0 else 0
        n = xyz.shape[0]
        g = self.buffers[back]
        for e in self.last_use[back]:          # readers of the old contents first
            self.est_stream.wait_event(e)
        self.last_use[back] = []
        if not xyz.is_cuda:
            with torch.cuda.stream(self.est_stream):
                self.stage_xyz[:n].copy_(xyz, non_blocking=True)
                self.stage_rgb[:n].copy_(rgb, non_blocking=True)
            xyz, rgb = self.stage_xyz[:n], self.stage_rgb[:n]
        view = type(g)(g.mean_op[:n], g.scale[:n], g.quat[:n], g.rgb[:n], g.normal[:n])
        self.est(xyz, rgb, mode=self.mode, mlp_blob=self.blob, out=view, stream=self.est_stream)
        ev = torch.cuda.Event()
        ev.record(self.est_stream)
        self.n[back], self.ready[back], self.version[back] = n, ev, version
        if self.front is None:
            ev.synchronize()
            self.est.check(n, self.est_stream)
            self.front = back
        else:
            self.pending = back

    def _gaussians(self, f):
        from .render import GaussianSet
        g, n = self.buffers[f], self.n[f]
        return GaussianSet(g.mean_op[:n], g.scale[:n], g.quat[:n], g.rgb[:n], g.normal[:n])

    def _render(self, h, check: bool):
        torch = self.torch
        from .render import Images
        st = self.streams[h["slot"]]
        with torch.cuda.stream(st):
            h["images"] = h.get("images") or Images(h["cams"], self.device)
            self.renderers[h["slot"]].render(self._gaussians(h["buffer"]), h["cams"], out=h["images"],
                                             check=check, stream=st)
            ev = torch.cuda.Event()
            ev.record(st)
        h["event"] = ev
        self.last_use[h["buffer"]].append(ev)

    def launch(self, slot: int, cams: list):
        self._promote()
        f = self.front
        if f is None:
            raise RuntimeError("no cloud published yet")
        h = dict(cams=cams, slot=slot, buffer=f, version=self.version[f])
        self.streams[slot].wait_event(self.ready[f])
        self._render(h, check=False)
        return h

    def query(self, h) -> bool:
        """True once the batch's images are final.  A batch whose keys
        overflowed the slot's capacity is rendered again (the renderer grows
        its buffers) before it reports completion."""
        from . import _lib
        from .render import p2e_bins_check
        if not h["event"].query():
            return False
        r = self.renderers[h["slot"]]
        st, k = p2e_bins_check(r.bins, self.streams[h["slot"]])
        if st == _lib.P2E_ERR_CAPACITY:
            # the batch's buffer may be re-estimated by now: render against
            # the current front buffer (the renderer grows its key buffers)
            self.rerenders += 1
            self._promote()
            h["buffer"], h["version"] = self.front, self.version[self.front]
            self.streams[h["slot"]].wait_event(self.ready[self.front])
            self._render(h, check=True)
            return False
        if st != _lib.P2E_OK:
            raise _lib.P2EError("p2e_sort_bin", st)
        return True

    def result(self, h, req: Request):
        if not self.keep_images:
            return None
        k = next(i for i, c in enumerate(h["cams"]) if c is req.camera)
        st = self.streams[h["slot"]]
        torch = self.torch
        with torch.cuda.stream(st):      # same stream as the buffers' allocation
            out = {key: val.clone() for key, val in h["images"].view(k).items()}
            # `last` is a position in the batch's sorted list: also give the
            # Gaussian it names, which does not depend on the batch
            _, vals = self.renderers[h["slot"]].bins.sorted()
            pos = out["last"].long()
            out["last_gaussian"] = torch.where(pos > 0, vals[(pos - 1).clamp(min=0)].long(),
                                               torch.full_like(pos, -1))
        st.synchronize()
        return out

    def release(self, h) -> None:
        h.pop("images", None)


def host_frames(cloud, frames: int) -> list:
    """Pinned (n, 4) float32 host tensors of the cloud's frames."""
    import torch
    out = []
    for k in range(frames):
        xyz, rgb = cloud.frame(k)
        a = torch.zeros((len(xyz), 4), dtype=torch.float32).pin_memory()
        b = torch.zeros((len(xyz), 4), dtype=torch.float32).pin_memory()
        a[:, :3] = torch.from_numpy(xyz)
        b[:, :3] = torch.from_numpy(rgb)
        out.append((a, b))
    return out


def run_load(seconds: float = 10.0, rate: float = 500.0, fps: float = 30.0, res=(1024, 2048),
             n_range=(300_000, 1_200_000), slots: int = 3, max_views: int = 8, seed: int = 5,
             learned: bool = True, frames: int = 16, deadline: float | None = None, tile: int = 16) -> dict:
    """Poisson viewpoint requests at ``rate``/s (square resolutions drawn
    uniformly from ``res``) against a moving humanoid cloud whose frames
    (point count swinging over ``n_range`` every 4 s) are uploaded from
    pinned host memory and estimated at ``fps``.  ``deadline`` (s): requests
    still queued that long after arrival are dropped (a display shows the
    latest pose).  Returns latency stats of the rendered requests and the
    number dropped."""
    import torch

    import scenes
    from . import mlp
    rng = np.random.default_rng(seed)
    blob = mlp.load_trained("cuda") if learned else None
    cloud = scenes.DynamicCloud(n_range, seed=seed, frames=frames)
    host = host_frames(cloud, frames)
    ex = GpuExecutor(n_range[1], slots, mlp_blob=blob, cfg={"tile": tile})
    sch = Scheduler(ex, slots=slots, max_views=max_views, deadline=deadline)
    center = np.array([0.0, 0.5, 0.0])
    # warm-up: both buffers estimated (the largest frame last, so the slots'
    # key buffers are sized for it), every slot renders full batches of
    # every resolution
    big = max(range(frames), key=cloud.count)
    for k in ((big + 1) % frames, big):
        ex.publish(*host[k], version=k)
        torch.cuda.synchronize()
        ex._promote()
    for s_ in range(slots):
        for r in res:
            h = ex.launch(s_, [scenes.sphere_camera(center, 2.5, rng, r, r) for _ in range(max_views)])
            torch.cuda.synchronize()
            while not ex.query(h):
                torch.cuda.synchronize()
            ex.release(h)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * seconds * 1.2) + 10))
    arrivals = arrivals[arrivals < seconds]
    cams = [scenes.sphere_camera(center, 2.5, rng, int(r), int(r)) for r in rng.choice(res, len(arrivals))]
    t0 = time.perf_counter()
    ai, fi = 0, 0
    reqs = []
    while True:
        now = time.perf_counter() - t0
        if now >= fi / fps and now < seconds:
            k = int(now * frames / cloud.period) % frames
            ex.publish(*host[k], version=fi)
            fi += 1
        while ai < len(arrivals) and arrivals[ai] <= now:
            reqs.append(sch.submit(cams[ai], arrival=t0 + arrivals[ai]))
            ai += 1
        sch.step()
        if ai >= len(arrivals) and not sch.pending and not sch.inflight:
            break
        time.sleep(0.00005)
    torch.cuda.synchronize()
    dropped = sum(1 for r in reqs if r.dropped)
    reqs = [r for r in reqs if not r.dropped]
    if not reqs:
        raise RuntimeError(f"every one of {dropped} requests was dropped")
    lat = np.array([r.latency for r in reqs]) * 1e3
    by_res = {}
    for r_ in res:
        m = np.array([int(r.camera["width"]) == int(r_) for r in reqs])
        if m.any():
            by_res[f"{r_}x{r_}"] = dict(n=int(m.sum()), p50_ms=float(np.percentile(lat[m], 50)),
                                      p99_ms=float(np.percentile(lat[m], 99)))
    px = sum(r.pixels for r in reqs)
    wall = max(r.done for r in reqs) - t0
    return dict(requests=len(reqs), p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                max_ms=float(lat.max()), within_10ms=float((lat < 10.0).mean()), by_resolution=by_res,
                batches=sch.next_bid, mean_views_per_batch=len(reqs) / max(sch.next_bid, 1),
                mpix_per_s=px / wall / 1e6, cloud_frames=fi, rerenders=ex.rerenders,
                path="learned" if blob is not None else "pca", rate=rate, seconds=seconds,
                points=list(n_range), fps=fps, tile=tile, dropped=dropped, deadline_ms=None if deadline is None else 1e3 * deadline)


def main(argv=None):
    ap = argparse.ArgumentParser(description="serve viewpoint requests against a dynamic cloud")
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--rate", type=float, default=500.0)
    ap.add_argument("--slots", type=int, default=3)
    ap.add_argument("--max-views", type=int, default=8)
    ap.add_argument("--pca", action="store_true")
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import json
    print(json.dumps(run_load(a.seconds, a.rate, slots=a.slots, max_views=a.max_views, learned=not a.pca)))


if __name__ == "__main__":
    main()

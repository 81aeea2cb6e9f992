"""Host-side serving policy with a fake executor and a fake clock: arrival
order, batch limits, slot and memory admission, deadline drops, latency
bookkeeping, and the dynamic cloud generator that feeds the server."""
import math

import numpy as np
import pytest

import scenes
from paper_2409_16504_gb300.serve import BYTES_PER_PIXEL, KEY_BYTES, Scheduler


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeExecutor:
    """Each batch takes ``per_mpix`` seconds per megapixel of fake device
    time from its launch."""

    def __init__(self, clock, per_mpix=1e-3):
        self.clock, self.per_mpix = clock, per_mpix
        self.launched = []

    def launch(self, slot, cams):
        px = sum(c["width"] * c["height"] for c in cams)
        h = dict(slot=slot, cams=list(cams), end=self.clock() + self.per_mpix * px / 1e6)
        self.launched.append(h)
        return h

    def query(self, h):
        return self.clock() >= h["end"]

    def result(self, h, req):
        return h["slot"]

    def release(self, h):
        h["released"] = True


def cam(w, h=None):
    return dict(width=w, height=h or w)


def test_arrival_order_and_batch_limit():
    clk = Clock()
    ex = FakeExecutor(clk)
    s = Scheduler(ex, slots=2, max_views=3, clock=clk)
    reqs = [s.submit(cam(64), arrival=0.0) for _ in range(8)]
    s.step()
    assert len(ex.launched) == 2                       # two slots
    assert [len(h["cams"]) for h in ex.launched] == [3, 3]
    assert [r.batch for r in reqs[:6]] == [0, 0, 0, 1, 1, 1]
    assert {h["slot"] for h in ex.launched} == {0, 1}
    assert len(s.pending) == 2
    clk.t = 1.0
    s.step()                                           # both complete, last batch goes out
    assert [r.batch for r in reqs[6:]] == [2, 2]
    clk.t = 2.0
    s.step()
    assert all(r.done is not None for r in reqs)
    assert sorted(r.rid for r in s.finished) == list(range(8))
    assert all(h.get("released") for h in ex.launched)


def test_slot_reuse_and_latency():
    clk = Clock()
    ex = FakeExecutor(clk, per_mpix=4e-3)              # 1024^2 -> ~4.2 ms
    s = Scheduler(ex, slots=1, max_views=1, clock=clk)
    a = s.submit(cam(1024), arrival=0.0)
    b = s.submit(cam(1024), arrival=0.001)
    s.step()
    assert a.batch == 0 and b.batch is None            # only one slot
    clk.t = 0.003
    s.step()
    assert a.done is None
    clk.t = 0.005
    s.step()
    assert a.done == 0.005 and b.batch == 1 and b.admitted == 0.005
    assert ex.launched[1]["slot"] == 0                 # the freed slot
    clk.t = 0.01
    s.step()
    assert b.done == 0.01
    assert math.isclose(a.latency, 0.005) and math.isclose(b.latency, 0.009)


def test_memory_admission():
    clk = Clock()
    ex = FakeExecutor(clk)
    per = int(256 * 256 * (BYTES_PER_PIXEL + 1.5 * KEY_BYTES))
    s = Scheduler(ex, slots=4, max_views=8, mem_budget=3 * per, clock=clk)
    with pytest.raises(ValueError):
        s.submit(cam(512))                             # one request above the whole budget
    rs = [s.submit(cam(256), arrival=0.0) for _ in range(5)]
    s.step()
    assert [len(h["cams"]) for h in ex.launched] == [3]    # budget caps the batch
    assert s.mem_in_use() == 3 * per
    assert rs[3].batch is None
    s.step()                                           # nothing fits until memory returns
    assert len(ex.launched) == 1
    clk.t = 1.0
    s.step()
    assert [len(h["cams"]) for h in ex.launched] == [3, 2]
    assert s.mem_in_use() == 2 * per


def test_oldest_request_blocks_while_it_does_not_fit():
    """Arrival order is kept: a large request waiting for memory is not
    overtaken by later small ones."""
    clk = Clock()
    ex = FakeExecutor(clk)
    small = int(128 * 128 * (BYTES_PER_PIXEL + 1.5 * KEY_BYTES))
    big = int(512 * 512 * (BYTES_PER_PIXEL + 1.5 * KEY_BYTES))
    s = Scheduler(ex, slots=4, max_views=8, mem_budget=big + small // 2, clock=clk)
    s.submit(cam(128), arrival=0.0)
    s.step()
    b = s.submit(cam(512), arrival=0.1)
    c = s.submit(cam(128), arrival=0.2)
    clk.t = 0.0
    s.step()                                           # big does not fit beside the first
    assert b.batch is None and c.batch is None
    clk.t = 1.0
    s.step()                                           # first done: big goes, small waits
    assert b.batch == 1 and c.batch is None
    clk.t = 2.0
    s.step()
    assert c.batch == 2


def test_deadline_drops_stale_requests():
    clk = Clock()
    ex = FakeExecutor(clk, per_mpix=10e-3)
    s = Scheduler(ex, slots=1, max_views=1, deadline=0.010, clock=clk)
    a = s.submit(cam(1024), arrival=0.0)
    b = s.submit(cam(1024), arrival=0.0)
    c = s.submit(cam(1024), arrival=0.008)
    s.step()
    clk.t = 0.0106                                     # a done; b is 10.6 ms old, c 2.6 ms
    s.step()
    assert a.done is not None and not a.dropped
    assert b.dropped and b.batch is None
    assert c.batch == 1 and not c.dropped
    assert len(ex.launched) == 2


def test_poisson_load_fake_device_all_complete():
    """A Poisson stream through the policy completes every request once, with
    latency at least the fake service time."""
    rng = np.random.default_rng(0)
    clk = Clock()
    ex = FakeExecutor(clk, per_mpix=1e-3)
    s = Scheduler(ex, slots=3, max_views=8, clock=clk)
    arr = np.cumsum(rng.exponential(1 / 500.0, 400))
    res = rng.choice([1024, 2048], 400)
    reqs, i = [], 0
    t = 0.0
    while i < len(arr) or s.pending or s.inflight:
        while i < len(arr) and arr[i] <= t:
            reqs.append(s.submit(cam(int(res[i])), arrival=float(arr[i])))
            i += 1
        s.step()
        t += 1e-4
        clk.t = t
    assert len(s.finished) == 400 and len({r.rid for r in s.finished}) == 400
    for r in reqs:
        assert r.done >= r.admitted >= r.arrival
        assert r.latency >= 1e-3 * r.pixels / 1e6 - 1e-12
    assert max(len(h["cams"]) for h in ex.launched) <= 8


# ------------------------------------------------------------ dynamic cloud
def test_dynamic_cloud_counts_and_surfaces():
    d = scenes.DynamicCloud((2000, 8000), seed=3, frames=8)
    counts = [d.count(k) for k in range(8)]
    assert min(counts) == 2000 and max(counts) == 8000
    assert counts[0] == 5000
    for k in (0, 3, 5):
        xyz, rgb = d.frame(k)
        assert xyz.shape == (counts[k], 3) and rgb.shape == (counts[k], 3)
        assert xyz.dtype == np.float32
        np.testing.assert_array_equal(rgb, d.rgb[: counts[k]])   # colours travel with the points
        prims = scenes.deform_primitives(d.prims, d.time_of(k))
        pid = d.pid[: counts[k]]
        x = xyz.astype(np.float64)
        for i, p in enumerate(prims):
            m = pid == i
            if p.kind != "cyl" or not m.any():
                continue
            ax = p.p1 - p.p0
            L = np.linalg.norm(ax)
            ax = ax / L
            rel = x[m] - p.p0
            tt = rel @ ax
            rad = np.linalg.norm(rel - tt[:, None] * ax, axis=1)
            # on the moved cylinder: side (radius r) or a cap (t = 0 or L),
            # within the 1e-3 position noise and float32 rounding
            dist = np.minimum(np.abs(rad - p.r), np.minimum(np.abs(tt), np.abs(tt - L)))
            assert dist.max() < 6e-3, (k, i, dist.max())
            assert tt.min() > -6e-3 and tt.max() < L + 6e-3


def test_limb_chain_stays_connected():
    prims = scenes.humanoid_primitives()
    for t in (0.0, 0.7, 1.9, 3.3):
        q = scenes.deform_primitives(prims, t)
        for side in range(2):
            b = 4 + 4 * side
            np.testing.assert_allclose(q[b].p1, q[b + 1].p0, atol=1e-12)      # elbow
            np.testing.assert_allclose(q[b + 2].p1, q[b + 3].p0, atol=1e-12)  # knee
            np.testing.assert_allclose(q[b].p0, prims[b].p0)                  # shoulder fixed
            for j in range(4):                                                # rigid segments
                assert math.isclose(np.linalg.norm(q[b + j].p1 - q[b + j].p0),
                                    np.linalg.norm(prims[b + j].p1 - prims[b + j].p0), rel_tol=1e-12)

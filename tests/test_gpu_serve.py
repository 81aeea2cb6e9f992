"""Serving loop on the GPU (continuous batching over the C-ABI).

* Every request's images are bit-identical (tolerance 0: rgb, normal, depth,
  alpha, and the Gaussian index of each pixel's last contributor) whether
  it is rendered alone or inside a batch of mixed resolutions: views of one
  batch share no arithmetic.
* Double buffering: a batch renders the cloud frame that was front when it
  was launched, even after later frames are estimated into the buffers;
  the estimate itself is deterministic (a second estimator reproduces it).
* A batch that overflows its slot's key capacity is rendered again and
  then matches a render with enough capacity.
* A short Poisson load over a moving cloud completes every request.
"""
import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu

PLANES = ("rgb", "normal", "depth", "alpha", "last_gaussian")


def _blob():
    from paper_2409_16504_gb300 import mlp
    return mlp.load_trained("cuda")


def _cloud(n, seed, t=0.0):
    from paper_2409_16504_gb300.estimate import cloud_tensors
    prims = scenes.deform_primitives(scenes.humanoid_primitives(), t)
    xyz, rgb, _, _ = scenes.humanoid_cloud(n, seed=seed, prims=prims)
    return cloud_tensors(xyz, rgb)


def _with_gaussian(view, renderer):
    """`last` is a position in the call's sorted list (it depends on the
    other views of the call); the Gaussian it names does not."""
    _, vals = renderer.bins.sorted()
    pos = view["last"].long()
    out = dict(view)
    out["last_gaussian"] = torch.where(pos > 0, vals[(pos - 1).clamp(min=0)].long(), torch.full_like(pos, -1))
    return out


def _alone(g, cam):
    from paper_2409_16504_gb300.render import Renderer
    r = Renderer(capacity=1 << 16)
    return _with_gaussian(r.render(g, [cam]).view(0), r)


def _same(a, b):
    for k in PLANES:
        assert torch.equal(a[k], b[k]), k
    assert ((a["last"] == 0) == (b["last"] == 0)).all()


def _finish(ex, h):
    torch.cuda.synchronize()
    while not ex.query(h):
        torch.cuda.synchronize()


def test_request_identical_alone_and_in_mix():
    from paper_2409_16504_gb300.serve import GpuExecutor, Scheduler
    ex = GpuExecutor(60_000, slots=2, mlp_blob=_blob(), keep_images=True, capacity=1 << 20)
    ex.publish(*_cloud(60_000, 3))
    sch = Scheduler(ex, slots=2, max_views=4)
    rng = np.random.default_rng(1)
    sizes = [(256, 256), (384, 256), (200, 328), (512, 512), (256, 256), (640, 480), (96, 96), (1024, 1024)]
    center = np.array([0.0, 0.5, 0.0])
    reqs = [sch.submit(scenes.sphere_camera(center, 2.5, rng, w, h)) for w, h in sizes]
    sch.drain()
    assert len(sch.finished) == len(reqs)
    assert max(sum(1 for r in reqs if r.batch == b) for b in range(sch.next_bid)) > 1
    g = ex._gaussians(ex.front)
    for r in reqs:
        assert r.images["rgb"].shape == (3, r.camera["height"], r.camera["width"])
        _same(r.images, _alone(g, r.camera))


def test_double_buffer_renders_the_launched_frame():
    from paper_2409_16504_gb300.estimate import LEARNED, PCA, Estimator
    from paper_2409_16504_gb300.serve import GpuExecutor
    blob = _blob()
    clouds = [_cloud(40_000, 10 + k, t=0.5 * k) for k in range(3)]
    ex = GpuExecutor(40_000, slots=3, mlp_blob=blob, capacity=1 << 20)
    rng = np.random.default_rng(2)
    center = np.array([0.0, 0.5, 0.0])
    cams = [[scenes.sphere_camera(center, 2.5, rng, 320, 240)] for _ in range(3)]
    ex.publish(*clouds[0], version=0)
    h0 = ex.launch(0, cams[0])
    ex.publish(*clouds[1], version=1)
    torch.cuda.synchronize()
    h1 = ex.launch(1, cams[1])
    ex.publish(*clouds[2], version=2)     # rewrites h0's buffer after h0 is done
    torch.cuda.synchronize()
    h2 = ex.launch(2, cams[2])
    hs = [h0, h1, h2]
    for h in hs:
        _finish(ex, h)
    assert [h["version"] for h in hs] == [0, 1, 2]
    est = Estimator(40_000)
    for k, h in enumerate(hs):
        g = est(*clouds[k], mode=LEARNED if blob is not None else PCA, mlp_blob=blob)
        _same(_with_gaussian(h["images"].view(0), ex.renderers[k]), _alone(g, cams[k][0]))


def test_capacity_overflow_rerenders():
    from paper_2409_16504_gb300.serve import GpuExecutor
    ex = GpuExecutor(30_000, slots=1, mlp_blob=None, capacity=1024)
    ex.publish(*_cloud(30_000, 4))
    rng = np.random.default_rng(3)
    cams = [scenes.sphere_camera(np.array([0.0, 0.5, 0.0]), 2.5, rng, 256, 256) for _ in range(2)]
    h = ex.launch(0, cams)
    _finish(ex, h)
    assert ex.rerenders == 1
    g = ex._gaussians(ex.front)
    for k in range(2):
        _same(_with_gaussian(h["images"].view(k), ex.renderers[0]), _alone(g, cams[k]))


def test_short_poisson_load_completes():
    from paper_2409_16504_gb300.serve import run_load
    r = run_load(seconds=1.0, rate=200.0, res=(256, 512), n_range=(50_000, 150_000), slots=2, max_views=4,
                 frames=4)
    assert r["requests"] > 100
    assert r["cloud_frames"] >= 25
    assert np.isfinite(r["p99_ms"]) and r["p50_ms"] > 0
    assert r["within_10ms"] > 0.5

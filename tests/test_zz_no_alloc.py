"""p2e_sort_bin_noalloc: the binning entry point for callers that may not
allocate device memory (for example code embedded in a host application
that owns the GPU memory budget, or a real-time loop where cudaMalloc could
stall).  Its scratch is a fixed array inside the library, shared by all
calls.  This test builds its own inputs, calls it twice in a row on
different views through the C ABI and checks every output against
p2e_sort_bin's (integer work: bit-exact), so stale scratch contents from
the first call would show in the second.  It also checks that sizes above
the stated limits are refused before anything runs."""
import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _scene():
    import scenes
    xyz, rgb, nrm, prims = scenes.humanoid_cloud(60_000, seed=11)
    sp = scenes.mean_spacing(60_000, prims)
    g = scenes.surface_gaussians(xyz, nrm, rgb, 1.13 * sp, np.random.default_rng(11))
    rng = np.random.default_rng(12)
    cams = [scenes.sphere_camera(xyz.mean(0), 2.5, rng, 512, 384) for _ in range(2)]
    return g, cams


def _noalloc(proj, n, cams, cfg, bins):
    from paper_2409_16504_gb300 import _lib
    from paper_2409_16504_gb300.render import _stream, make_cameras, make_config
    ca, cf, ps = make_cameras(cams), make_config(cfg), proj.c_struct()
    return _lib.load().p2e_sort_bin_noalloc(C.byref(ps), n, ca, len(cams), C.byref(cf),
                                            C.byref(bins.struct), _stream())


def test_noalloc_sort_bin_matches_sort_bin_twice():
    from paper_2409_16504_gb300 import Bins, GaussianSet, Projected, p2e_bins_check, p2e_project, p2e_sort_bin
    from paper_2409_16504_gb300.render import DEFAULT_CONFIG, total_tiles
    g, cams = _scene()
    gs = GaussianSet.from_numpy(g)
    cfg = dict(DEFAULT_CONFIG)
    for cam in cams:                       # two calls in a row, different views
        tt = total_tiles([cam], cfg["tile"])
        proj = Projected(gs.n)
        p2e_project(gs, [cam], cfg, proj)
        ref = Bins(gs.n, tt, 1 << 19)
        p2e_sort_bin(proj, gs.n, [cam], cfg, ref)
        st, k_ref = p2e_bins_check(ref)
        assert st == 0 and k_ref > 0
        out = Bins(gs.n, tt, 1 << 19)
        out.struct.scratch = None          # ignored by the entry point
        out.struct.scratch_bytes = 0
        assert _noalloc(proj, gs.n, [cam], cfg, out) == 0
        st, k = p2e_bins_check(out)
        assert st == 0 and k == k_ref
        assert out.struct.result == ref.struct.result
        rk, rv = ref.sorted()
        ok, ov = out.sorted()
        assert torch.equal(ok[:k], rk[:k]) and torch.equal(ov[:k], rv[:k])
        assert torch.equal(out.ranges, ref.ranges)
        # the work list holds the same non-empty tiles, longest class first;
        # the order inside a length class comes from atomics and is free
        nw = int(ref.tile_work[0])
        assert int(out.tile_work[0]) == nw
        a = out.tile_work[2: 2 + nw].cpu().numpy()
        b = ref.tile_work[2: 2 + nw].cpu().numpy()
        assert sorted(a.tolist()) == sorted(b.tolist())
        lens = (ref.ranges[:, 1] - ref.ranges[:, 0]).cpu().numpy()
        cls = np.floor(np.log2(lens[a].astype(np.float64)))
        assert (np.diff(cls) <= 0).all()


def test_noalloc_rejects_sizes_beyond_limit():
    from paper_2409_16504_gb300 import Bins, Projected, _lib
    from paper_2409_16504_gb300.render import DEFAULT_CONFIG
    import scenes
    cam = scenes.look_at_camera((0, 0, -3), (0, 0, 0), (0, -1, 0), 60, 64, 64)
    proj = Projected(16)
    big = Bins(16, 16, 1 << 10)
    big.struct.capacity = _lib.NOALLOC_MAX_CAPACITY + 1
    assert _noalloc(proj, 16, [cam], DEFAULT_CONFIG, big) == _lib.P2E_ERR_INVALID_ARG
    small = Bins(16, 16, 1 << 10)
    assert _noalloc(proj, _lib.NOALLOC_MAX_N + 1, [cam], DEFAULT_CONFIG, small) == _lib.P2E_ERR_INVALID_ARG

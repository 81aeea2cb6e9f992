"""GPU parity of the forward path (project, sort_bin, render) against the
FP64 oracle: binning bit-exact, images within 1e-4 max-abs per channel."""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import (TOL, cfg1_scene, compare_images, gpu_proj_view, gpu_render,
                        humanoid_scene, random_scene)

pytestmark = pytest.mark.gpu


def _check_projection(r, g, cams, cfg=None):
    n = len(g["mean"])
    for v, cam in enumerate(cams):
        p = oracle.project(g, cam, cfg)
        gp = gpu_proj_view(r, v, n)
        np.testing.assert_array_equal(gp["ntiles"], p["ntiles"])
        vis = p["vis"].astype(bool)
        B = (cfg or {}).get("tile", 16)
        # tiles exact; pixel bounds a superset of the exact ones
        np.testing.assert_array_equal(gp["prect"][vis] // B, p["trect"][vis])
        pr, gr = p["prect"][vis], gp["prect"][vis]
        assert (gr[:, 0] <= pr[:, 0]).all() and (gr[:, 1] >= pr[:, 1]).all()
        assert (gr[:, 2] <= pr[:, 2]).all() and (gr[:, 3] >= pr[:, 3]).all()
        # the depth key is fp32 of the double depth: bit-exact for every Gaussian
        np.testing.assert_array_equal(gp["zkey"].view(np.uint32), p["zkey"].view(np.uint32))
        np.testing.assert_allclose(gp["uv"][vis], p["uv"][vis], atol=2e-5, rtol=0)
        np.testing.assert_allclose(gp["conic"][vis], p["conic"][vis], rtol=2e-5,
                                   atol=2e-5 * np.abs(p["conic"][vis]).max())


def _check_bins(r, g, cams, cfg=None):
    projs = [oracle.project(g, c, cfg) for c in cams]
    keys, vals, ranges = oracle.bin_keys(projs, cams, cfg)
    assert r.n_keys == len(keys)
    gk, gv = r.bins.sorted()
    K = len(keys)
    np.testing.assert_array_equal(gk[:K].cpu().numpy().view(np.uint64), keys)
    np.testing.assert_array_equal(gv[:K].cpu().numpy().view(np.uint32), vals)
    np.testing.assert_array_equal(r.bins.ranges[: len(ranges)].cpu().numpy().view(np.uint32), ranges)
    return keys, vals, ranges


def _check_images(r, out, g, cams, cfg=None, tol=TOL, max_flag_mismatch=None):
    cfg = {**oracle.DEFAULT_CFG, **(cfg or {})}
    keys, vals, ranges = _check_bins(r, g, cams, cfg)
    base = 0
    errs = []
    for v, cam in enumerate(cams):
        orc = oracle.render(g, cam, cfg)
        tx, ty = oracle.tiles_of(cam, cfg["tile"])
        errs.append(compare_images(out.view(v), orc, tol, vals=vals, ranges=ranges,
                                   tile=cfg["tile"], tile_base=base, tiles_x=tx,
                                   max_flag_mismatch=max_flag_mismatch))
        base += tx * ty
    return errs


def test_cfg1_sphere_128():
    """The 4096-point sphere: every pixel within 1e-4, knife-edge pixels
    included (the oracle flags ~8 of 16384; fp32 takes the same decisions
    there, so none is excluded in effect)."""
    g, cam = cfg1_scene()
    r, out = gpu_render(g, [cam])
    _check_projection(r, g, [cam])
    errs = _check_images(r, out, g, [cam], max_flag_mismatch=0)
    assert np.count_nonzero(out.view(0)["alpha"].cpu().numpy()) > 1000
    print("cfg1 max errors", errs)


@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("W,H,n", [(100, 70, 3001), (37, 129, 777)])
def test_random_ragged(tile, W, H, n):
    g, cam = random_scene(10 + tile + W, n, W, H)
    cfg = {"tile": tile, "bg": (0.1, 0.2, 0.3)}
    r, out = gpu_render(g, [cam], cfg)
    _check_projection(r, g, [cam], cfg)
    _check_images(r, out, g, [cam], cfg)


def test_multiview_mixed_resolution():
    g, _ = random_scene(3, 2500, 64, 64)
    import scenes
    cams = [scenes.look_at_camera(e, (0, 0, 0), (0, 1, 0), 50, w, h)
            for e, w, h in (((0.1, -0.2, -2.0), 64, 48), ((1.5, 0.3, -1.4), 128, 128),
                            ((-1.8, 0.5, 0.9), 96, 80))]
    r, out = gpu_render(g, cams)
    _check_projection(r, g, cams)
    _check_images(r, out, g, cams)


def test_tile_size_invariance():
    g, cam = random_scene(4, 2000, 96, 64)
    imgs = []
    for t in (8, 16, 32):
        r, out = gpu_render(g, [cam], {"tile": t})
        imgs.append(out.view(0)["rgb"].cpu().numpy())
    # same splats in the same order per pixel; only the grouping of the
    # partial sums differs with the tile size
    np.testing.assert_allclose(imgs[0], imgs[1], atol=2e-6)
    np.testing.assert_allclose(imgs[0], imgs[2], atol=2e-6)


def test_empty_and_fully_culled():
    g, cam = random_scene(5, 200, 48, 32)
    bg = (0.3, 0.6, 0.9)
    empty = {k: v[:0] for k, v in g.items()}
    r, out = gpu_render(empty, [cam], {"bg": bg})
    rgb = out.view(0)["rgb"].cpu().numpy()
    assert np.allclose(rgb, np.asarray(bg, np.float32)[:, None, None], atol=0)
    assert r.n_keys == 0
    g["mean"][:] = (0, 0, -2.5)  # all behind the camera
    r, out = gpu_render(g, [cam], {"bg": bg})
    assert r.n_keys == 0
    assert (out.view(0)["alpha"].cpu().numpy() == 0).all()


def test_zero_opacity_background():
    g, cam = random_scene(6, 500, 64, 48)
    g["opacity"][:] = 0
    r, out = gpu_render(g, [cam], {"bg": (0.25, 0.5, 0.75)})
    v = out.view(0)
    assert (v["rgb"].cpu().numpy() == np.float32([0.25, 0.5, 0.75])[:, None, None]).all()
    assert (v["alpha"].cpu().numpy() == 0).all()


def test_capacity_overflow_reported_and_recovered():
    from paper_2409_16504_gb300 import GaussianSet, Renderer, p2e_bins_check
    from paper_2409_16504_gb300._lib import P2E_ERR_CAPACITY
    g, cam = random_scene(7, 3000, 128, 96)
    gs = GaussianSet.from_numpy(g)
    r = Renderer(capacity=64)
    out = r.render(gs, [cam], check=False)
    st, k = p2e_bins_check(r.bins)
    assert st == P2E_ERR_CAPACITY and k > 64
    out = r.render(gs, [cam])            # grows and re-renders
    torch.cuda.synchronize()
    assert r.capacity >= k
    _check_images(r, out, g, [cam])


def test_invalid_arguments_rejected_before_launch():
    from paper_2409_16504_gb300 import GaussianSet, P2EError, Renderer
    g, cam = random_scene(8, 100, 32, 32)
    gs = GaussianSet.from_numpy(g)
    with pytest.raises(P2EError):
        Renderer({"tile": 12}).render(gs, [cam])
    bad = dict(cam)
    bad["width"] = 0
    with pytest.raises(P2EError):
        Renderer().render(gs, [bad])
    bad = dict(cam)
    bad["near"] = -1.0
    with pytest.raises(P2EError):
        Renderer().render(gs, [bad])


def test_full_size_humanoid_800k_1024():
    """800K points, 1024^2: bit-exact keys/ranges, images within 1e-4 on
    every pixel (the oracle renders the whole frame; it flags ~190 knife-edge
    pixels, on which fp32 takes the same decisions)."""
    g, cam = humanoid_scene(800_000, 1024, 1024)
    r, out = gpu_render(g, [cam], capacity=1 << 21)
    _check_projection(r, g, [cam])
    errs = _check_images(r, out, g, [cam], max_flag_mismatch=0)
    print("800K max errors", errs)


def _chain_info(r):
    """(chained schedule in use, multi-segment tiles run by one warp per
    block) from the item table the compositing leaves in the free value
    buffer: word 0 and word 2 n_work + 3."""
    v = r.bins.vals[1 - r.bins.struct.result]
    n_work = int(r.bins.tile_work[0].item())
    return int(v[0].item()), int(v[2 * n_work + 3].item())


def test_segment_chains_schedule_independent():
    """Long tile lists are split into segments combined by the 'over' rule.
    Chained across warps (states in the free key buffers) or run by one warp
    per pixel block (P2E_SCHEDULE_PER_BLOCK): the arithmetic is the same,
    the images are bit-identical."""
    from paper_2409_16504_gb300 import GaussianSet, Renderer
    g, cam = humanoid_scene(300_000, 1024, 1024, seed=4)
    gs = GaussianSet.from_numpy(g)
    big = Renderer(capacity=1 << 22)
    a = big.render(gs, [cam])
    lengths = (big.bins.ranges.view(-1, 2)[:, 1] - big.bins.ranges.view(-1, 2)[:, 0]).cpu().numpy()
    assert lengths.max() > 3 * 1024  # several segments per tile
    one = Renderer({"schedule": 1}, capacity=1 << 22)
    b = one.render(gs, [cam])
    torch.cuda.synchronize()
    assert _chain_info(big) == (1, 0)
    assert _chain_info(one)[0] == 0
    for key in ("rgb", "normal", "depth", "alpha", "last"):
        assert torch.equal(getattr(a, key), getattr(b, key)), key


def test_chaining_mixed_tile_by_tile_when_states_run_short():
    """A field of small splats whose tile lists all run just past one
    segment: two state slots per tile need about twice the key count, so at
    a capacity equal to the key count the longest tiles chain and the rest
    run one warp per block, in the same launch; the images are
    bit-identical to both pure schedules."""
    import scenes
    from paper_2409_16504_gb300 import GaussianSet, Renderer
    rng = np.random.default_rng(11)
    n, W = 240_000, 256
    cam = scenes.look_at_camera((0.0, 0.0, -2.0), (0, 0, 0), (0, 1, 0), 55, W, W)
    mean = np.stack([rng.uniform(-1.0, 1.0, n), rng.uniform(-1.0, 1.0, n), rng.uniform(-0.05, 0.05, n)], 1)
    g = dict(mean=mean.astype(np.float32),
             scale=np.full((n, 3), 0.004, np.float32),
             quat=rng.standard_normal((n, 4)).astype(np.float32),
             opacity=rng.uniform(0.05, 0.4, n).astype(np.float32),
             rgb=rng.random((n, 3)).astype(np.float32),
             normal=rng.standard_normal((n, 3)).astype(np.float32))
    gs = GaussianSet.from_numpy(g)
    big = Renderer(capacity=1 << 21)
    a = big.render(gs, [cam])
    torch.cuda.synchronize()
    k = big.n_keys
    lengths = (big.bins.ranges.view(-1, 2)[:, 1] - big.bins.ranges.view(-1, 2)[:, 0]).cpu().numpy()
    multi = lengths[lengths > 1024]
    need = int(np.ceil(multi / 1024.0).sum()) * 1024
    assert need > 1.1 * k, (need, k)  # the scene must make the states run short
    mixed = Renderer(capacity=k)
    b = mixed.render(gs, [cam])
    one = Renderer({"schedule": 1}, capacity=1 << 21)
    c = one.render(gs, [cam])
    torch.cuda.synchronize()
    assert _chain_info(big) == (1, 0)
    ch, alone = _chain_info(mixed)
    assert ch == 1 and 0 < alone < len(multi), (ch, alone, len(multi))
    print(f"mixed schedule: {len(multi) - alone} of {len(multi)} multi-segment tiles chained, {k} keys")
    for key in ("rgb", "normal", "depth", "alpha", "last"):
        assert torch.equal(getattr(a, key), getattr(b, key)), key
        assert torch.equal(getattr(a, key), getattr(c, key)), key


def test_very_long_tile_list_chains():
    """One 16 x 16 tile holding 300K faint splats (the stop rule never
    fires, so every one of its 293 segments is walked and chained): the
    chained images are bit-identical to one warp per block."""
    import scenes
    from paper_2409_16504_gb300 import GaussianSet, Renderer
    rng = np.random.default_rng(5)
    n = 300_000
    cam = scenes.look_at_camera((0.0, 0.0, -2.0), (0, 0, 0), (0, 1, 0), 55, 16, 16)
    mean = np.stack([rng.uniform(-1.0, 1.0, n), rng.uniform(-1.0, 1.0, n), rng.uniform(-0.2, 0.2, n)], 1)
    g = dict(mean=mean.astype(np.float32),
             scale=np.full((n, 3), 0.04, np.float32),
             quat=rng.standard_normal((n, 4)).astype(np.float32),
             opacity=rng.uniform(0.004, 0.0055, n).astype(np.float32),  # above the floor near the centre only
             rgb=rng.random((n, 3)).astype(np.float32),
             normal=rng.standard_normal((n, 3)).astype(np.float32))
    gs = GaussianSet.from_numpy(g)
    a_r = Renderer(capacity=1 << 20)
    a = a_r.render(gs, [cam])
    b_r = Renderer({"schedule": 1}, capacity=1 << 20)
    b = b_r.render(gs, [cam])
    torch.cuda.synchronize()
    assert a_r.n_keys > 257 * 1024, a_r.n_keys
    assert _chain_info(a_r) == (1, 0) and _chain_info(b_r)[0] == 0
    assert float((a.alpha < 0.9999).float().mean()) > 0.5  # most pixels stay open to the end of the list
    for key in ("rgb", "normal", "depth", "alpha", "last"):
        assert torch.equal(getattr(a, key), getattr(b, key)), key


def test_chained_schedule_fits_at_the_benchmark_capacity():
    """At the benchmark's key capacity (2x the first view's keys + 4096) and
    tile sizes (8 px for the frames, 16 px as the library's default) every
    multi-segment tile of the 800K-point humanoid's views chains, for 24
    camera positions on the 2.5 m sphere."""
    import scenes
    from paper_2409_16504_gb300 import GaussianSet, Renderer
    g, cam = humanoid_scene(800_000, 1024, 1024)
    gs = GaussianSet.from_numpy(g)
    c = np.asarray(g["mean"], np.float64).mean(0)
    rng = np.random.default_rng(102)
    cams = [scenes.sphere_camera(c, 2.5, rng, 1024, 1024) for _ in range(24)]
    for tile in (8, 16):
        r = Renderer({"tile": tile}, capacity=1 << 22)
        r.render(gs, [cams[0]])
        r = Renderer({"tile": tile}, capacity=int(r.n_keys * 2.0) + 4096)
        keys = []
        for cam in cams:
            r.render(gs, [cam])
            torch.cuda.synchronize()
            keys.append(r.n_keys)
            assert _chain_info(r) == (1, 0), (tile, r.n_keys, r.capacity, _chain_info(r))
        print(f"tile {tile}: keys per view {min(keys)} .. {max(keys)} at capacity {r.capacity}: all chained")


def test_depth_first_and_full_key_binning_agree():
    """Binning sorts the Gaussians by depth first and then the tile keys by
    tile only when the key buffers hold an entry per Gaussian; with fewer
    entries it sorts all key bits.  Both give the same sorted keys, values,
    tile ranges and images, and both match the oracle's binning."""
    from paper_2409_16504_gb300 import GaussianSet, Renderer
    g, cam = humanoid_scene(120_000, 512, 512, seed=7)
    cam = dict(cam, cx=cam["cx"] - 0.5 * cam["width"])  # half the figure off screen
    gs = GaussianSet.from_numpy(g)
    big = Renderer(capacity=1 << 20)
    a = big.render(gs, [cam])
    k = big.n_keys
    n = len(g["mean"])
    assert 1000 < k < n  # the small buffers cannot take the depth sort
    small = Renderer(capacity=k)
    b = small.render(gs, [cam])
    torch.cuda.synchronize()
    ka, va = big.bins.sorted()
    kb, vb = small.bins.sorted()
    assert torch.equal(ka[:k], kb[:k]) and torch.equal(va[:k], vb[:k])
    tt = big.bins.ranges.numel()
    assert torch.equal(big.bins.ranges[:tt], small.bins.ranges[:tt])
    for key in ("rgb", "normal", "depth", "alpha", "last"):
        assert torch.equal(getattr(a, key), getattr(b, key)), key
    _check_bins(big, g, [cam])
    _check_bins(small, g, [cam])

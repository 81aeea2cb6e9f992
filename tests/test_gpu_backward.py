"""GPU backward (p2e_render_backward) against the oracle's exact FP64
gradient, on multi-view scenes with ragged image sizes.

Tolerance: per parameter array, max |gpu - oracle| <= 1e-4 * max |oracle|
+ 1e-6.  The fp32 path recomputes each pixel's final transmittance front
to back over its tile list, recovers T backwards by division, accumulates
per-splat sums with float atomics in arbitrary order and evaluates the
chain rule in fp32; each term carries a relative error of order 1e-6, far
inside that bound.  The opaque-surface case (most covered pixels end with
T near the 1e-4 cutoff) is where recovering T from the fp32 alpha image
would lose ~2.5e-4 relative accuracy.
"""
import numpy as np
import pytest
import torch

import oracle
import scenes
from gpu_common import random_scene

pytestmark = pytest.mark.gpu


def _cams():
    return [scenes.look_at_camera((0.1, -0.2, -2.0), (0, 0, 0), (0, 1, 0), 50, 61, 47),
            scenes.look_at_camera((1.4, 0.4, -1.3), (0, 0, 0), (0, 1, 0), 45, 48, 40)]


def _upstream(cams, g, cfg, seed):
    rng = np.random.default_rng(seed)
    ups = []
    for cam in cams:
        u = rng.standard_normal((8, cam["height"], cam["width"]))
        flag = oracle.render(g, cam, cfg)["flag"]
        u[:, flag] = 0.0  # knife-edge pixels: decisions may differ between fp32 and fp64
        ups.append(u)
    return ups


def _gpu_grads(g, cams, cfg, ups, lengths=None):
    """The GPU gradients; ``lengths`` (a list) receives the tile list lengths."""
    from paper_2409_16504_gb300 import GaussianSet, Renderer, p2e_render_backward
    gs = GaussianSet.from_numpy(g)
    r = Renderer(cfg, capacity=1 << 20)
    img = r.render(gs, cams)
    if lengths is not None:
        rg = r.bins.ranges.cpu().numpy().astype(np.int64)
        lengths.extend((rg[:, 1] - rg[:, 0]).tolist())

    def planes(k0, k1):
        return torch.from_numpy(np.concatenate([u[k0:k1].reshape(-1) for u in ups]).astype(np.float32)).cuda()

    d = p2e_render_backward(gs, r.proj, r.bins, cams, cfg, img.alpha, img.last,
                            d_rgb=planes(0, 3), d_normal=planes(3, 6), d_depth=planes(6, 7),
                            d_alpha=planes(7, 8))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in d.items()}


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_backward_matches_oracle(tile):
    g, _ = random_scene(21 + tile, 400, 64, 64)
    cams = _cams()
    cfg = {**oracle.DEFAULT_CFG, "tile": tile, "bg": (0.2, 0.1, 0.3)}
    ups = _upstream(cams, g, cfg, tile)
    ref = oracle.render_grad(g, cams, ups, cfg)
    got = _gpu_grads(g, cams, cfg, ups)
    for k in oracle.GRAD_KEYS:
        err = np.abs(got[k] - ref[k]).max()
        tol = 1e-4 * np.abs(ref[k]).max() + 1e-6
        assert err <= tol, f"{k}: max err {err:.3g} > {tol:.3g} (max |ref| {np.abs(ref[k]).max():.3g})"
        assert np.abs(ref[k]).max() > 0


def _opaque_scene():
    from gpu_common import humanoid_scene
    g, _ = humanoid_scene(20_000, 96, 96, seed=9)
    c = g["mean"].mean(0)
    cams = [scenes.look_at_camera(tuple(c + np.array(e)), tuple(c), (0, -1, 0), 45, 96, 96)
            for e in ((0.0, 0.3, -1.2), (0.9, -0.2, 0.8))]
    return g, cams


@pytest.mark.parametrize("tile", [8, 16])
def test_backward_opaque_humanoid(tile):
    """20K-point humanoid of opaque surface splats (opacity 0.9), two close
    views at 96^2: about a quarter of the pixels end with T < 1e-3, with up
    to ~130 contributing splats per pixel."""
    g, cams = _opaque_scene()
    cfg = {**oracle.DEFAULT_CFG, "tile": tile, "bg": (0.2, 0.1, 0.3)}
    sat = [float(((1 - oracle.render(g, c, cfg)["alpha"]) < 1e-3).mean()) for c in cams]
    assert min(sat) > 0.2, sat
    ups = _upstream(cams, g, cfg, 40 + tile)
    ref = oracle.render_grad(g, cams, ups, cfg)
    got = _gpu_grads(g, cams, cfg, ups)
    for k in oracle.GRAD_KEYS:
        err = np.abs(got[k] - ref[k]).max()
        tol = 1e-4 * np.abs(ref[k]).max() + 1e-6
        print(f"{k}: max err {err:.3g}, tol {tol:.3g}")
        assert err <= tol, f"{k}: max err {err:.3g} > {tol:.3g} (max |ref| {np.abs(ref[k]).max():.3g})"
        assert np.abs(ref[k]).max() > 0


@pytest.mark.parametrize("tile", [8, 16])
def test_backward_segments_match_whole_walks(tile):
    """Tile lists longer than 4 x tile^2 splats are walked as parallel
    segments (schedule AUTO) or whole (PER_BLOCK): the opaque humanoid has
    such lists, and both schedules agree with each other to fp32 rounding
    order (1e-5 relative) and with the oracle (1e-4)."""
    g, cams = _opaque_scene()
    cfg = {**oracle.DEFAULT_CFG, "tile": tile, "bg": (0.2, 0.1, 0.3)}
    ups = _upstream(cams, g, cfg, 60 + tile)
    lens = []
    seg = _gpu_grads(g, cams, {**cfg, "schedule": 0}, ups, lengths=lens)
    lens = np.array(lens)
    assert (lens > 4 * tile * tile).sum() >= 4, lens.max()
    whole = _gpu_grads(g, cams, {**cfg, "schedule": 1}, ups)
    ref = oracle.render_grad(g, cams, ups, cfg)
    for k in oracle.GRAD_KEYS:
        scale = np.abs(ref[k]).max()
        assert np.abs(seg[k] - whole[k]).max() <= 1e-5 * scale + 1e-7, k
        assert np.abs(seg[k] - ref[k]).max() <= 1e-4 * scale + 1e-6, k


def test_backward_segments_on_a_very_long_list():
    """Thousands of splats stacked on one 8-px tile (the list spans dozens of
    256-splat segments, most pixels saturate early): segmented gradients
    equal the oracle's."""
    rng = np.random.default_rng(5)
    n = 6000
    cam = scenes.look_at_camera((0.0, 0.0, -2.0), (0, 0, 0), (0, 1, 0), 50, 24, 20)
    g = dict(mean=np.column_stack([rng.uniform(-0.04, 0.04, n), rng.uniform(-0.04, 0.04, n),
                                   rng.uniform(-0.5, 0.5, n)]),
             scale=rng.uniform(0.008, 0.04, (n, 3)), quat=rng.standard_normal((n, 4)),
             opacity=rng.uniform(0.02, 0.3, n), rgb=rng.uniform(0, 1, (n, 3)),
             normal=rng.standard_normal((n, 3)))
    g["normal"] /= np.linalg.norm(g["normal"], axis=1, keepdims=True)
    g = {k: v.astype(np.float32) for k, v in g.items()}
    cfg = {**oracle.DEFAULT_CFG, "tile": 8}
    ups = _upstream([cam], g, cfg, 77)
    lens = []
    got = _gpu_grads(g, [cam], cfg, ups, lengths=lens)
    assert max(lens) > 20 * 256, max(lens)
    ref = oracle.render_grad(g, [cam], ups, cfg)
    for k in oracle.GRAD_KEYS:
        err = np.abs(got[k] - ref[k]).max()
        tol = 1e-4 * np.abs(ref[k]).max() + 1e-6
        assert err <= tol, f"{k}: max err {err:.3g} > {tol:.3g}"


def test_autograd_function_equals_direct_call():
    from paper_2409_16504_gb300 import GaussianSet, render_differentiable
    g, _ = random_scene(31, 300, 48, 48)
    cams = _cams()
    gs = GaussianSet.from_numpy(g)
    params = [t.clone().requires_grad_(True) for t in (gs.mean_op, gs.scale, gs.quat, gs.rgb, gs.normal)]
    rgb, nrm, dep, alp = render_differentiable(*params, cams)
    rng = np.random.default_rng(3)
    w = [torch.from_numpy(rng.standard_normal(t.shape).astype(np.float32)).cuda() for t in (rgb, nrm, dep, alp)]
    loss = sum((a * b).sum() for a, b in zip((rgb, nrm, dep, alp), w))
    loss.backward()
    ups = []
    off = 0
    for cam in cams:
        H, W = cam["height"], cam["width"]
        n = H * W
        u = np.concatenate([w[0][3 * off:3 * off + 3 * n].cpu().numpy().reshape(3, H, W),
                            w[1][3 * off:3 * off + 3 * n].cpu().numpy().reshape(3, H, W),
                            w[2][off:off + n].cpu().numpy().reshape(1, H, W),
                            w[3][off:off + n].cpu().numpy().reshape(1, H, W)])
        ups.append(u.astype(np.float64))
        off += n
    direct = _gpu_grads(g, cams, oracle.DEFAULT_CFG, ups)
    np.testing.assert_allclose(params[0].grad[:, :3].cpu().numpy(), direct["mean"], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(params[0].grad[:, 3].cpu().numpy(), direct["opacity"], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(params[2].grad.cpu().numpy(), direct["quat"], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(params[3].grad[:, :3].cpu().numpy(), direct["rgb"], rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_backward_probe_counts(tile):
    """The work counters of the backward kernel's probe: its contributing
    (pixel, splat) pairs are exactly the oracle's per-pixel contributor
    counts summed (a scene with no knife-edge pixel), every reduction
    carries 1..32 of them, and every contributing pair was evaluated."""
    import ctypes as C
    from paper_2409_16504_gb300 import GaussianSet, Renderer, _lib, p2e_render_backward
    g, _ = random_scene(21, 400, 64, 64)
    cams = _cams()
    cfg = {**oracle.DEFAULT_CFG, "tile": tile}
    refs = [oracle.render(g, c, cfg) for c in cams]
    assert sum(int(r["flag"].sum()) for r in refs) == 0
    want = sum(int(r["ncontrib"].sum()) for r in refs)
    gs = GaussianSet.from_numpy(g)
    r = Renderer(cfg, capacity=1 << 16)
    img = r.render(gs, cams)
    n_pix = sum(c["height"] * c["width"] for c in cams)
    d_rgb = torch.ones(3 * n_pix, device="cuda")
    count = torch.zeros(3, dtype=torch.int64, device="cuda")
    lib = _lib.load()
    p = _lib.P2EKernelProbe(None, None, count.data_ptr())
    _lib.check("p2e_set_kernel_probe", lib.p2e_set_kernel_probe(_lib.P2E_PROBE_BLEND_BWD, C.byref(p)))
    try:
        p2e_render_backward(gs, r.proj, r.bins, cams, cfg, img.alpha, img.last, d_rgb=d_rgb)
        torch.cuda.synchronize()
    finally:
        lib.p2e_set_kernel_probe(_lib.P2E_PROBE_BLEND_BWD, None)
    n_eval, n_contrib, n_red = (int(v) for v in count.cpu())
    assert n_contrib == want
    assert n_eval >= n_contrib
    assert n_contrib <= 32 * n_red and n_red <= n_contrib


@pytest.mark.parametrize("tile", [8, 16])
def test_backward_empty_culled_and_unreached(tile):
    """Degenerate inputs of the backward: no Gaussians, every Gaussian
    culled (no keys, no work tiles), and splats that all fall below the
    alpha floor (lists that no pixel walks: every walk end is the list
    start).  The call succeeds and every gradient is zero."""
    from paper_2409_16504_gb300 import GaussianSet, Renderer, p2e_render_backward
    g, _ = random_scene(7, 300, 40, 40)
    cams = _cams()
    cfg = {**oracle.DEFAULT_CFG, "tile": tile}
    n_pix = sum(c["height"] * c["width"] for c in cams)
    faint = {k: v.copy() for k, v in g.items()}
    faint["opacity"][:] = 1e-4  # alpha <= 1e-4 < 1/255 everywhere
    culled = {k: v.copy() for k, v in g.items()}
    culled["mean"][:] = (0.0, 0.0, -2.5)  # behind both cameras
    empty = {k: v[:0] for k, v in g.items()}
    for name, scene in (("empty", empty), ("culled", culled), ("faint", faint)):
        gs = GaussianSet.from_numpy(scene)
        r = Renderer(cfg, capacity=1 << 16)
        img = r.render(gs, cams)
        d = p2e_render_backward(gs, r.proj, r.bins, cams, cfg, img.alpha, img.last,
                                d_rgb=torch.ones(3 * n_pix, device="cuda"),
                                d_normal=torch.ones(3 * n_pix, device="cuda"),
                                d_depth=torch.ones(n_pix, device="cuda"), d_alpha=torch.ones(n_pix, device="cuda"))
        torch.cuda.synchronize()
        if name == "faint":
            assert r.n_keys > 0
        for k, v in d.items():
            assert v.shape[0] == len(scene["mean"]), (name, k)
            assert not v.any(), (name, k)

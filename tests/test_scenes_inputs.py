"""The input degradations of the training and robustness data (scenes):
10-bit voxelisation with merging, its alpha coarsening, and subsampling."""
import numpy as np

import scenes


def test_quantize_grid_merge_and_colours():
    rng = np.random.default_rng(0)
    xyz = rng.uniform(-0.4, 0.6, (5000, 3)).astype(np.float32)
    rgb = rng.random((5000, 3)).astype(np.float32)
    for alpha in (1.0, 0.5, 0.25):
        q, c = scenes.quantize_cloud(xyz, rgb, alpha=alpha)
        lo, hi = xyz.astype(np.float64).min(0), xyz.astype(np.float64).max(0)
        cen, s = 0.5 * (lo + hi), 2.0 / (hi - lo).max()
        u = (q.astype(np.float64) - cen) * s * 512 * alpha       # voxel units: integers
        assert np.abs(u - np.round(u)).max() < 1e-3
        assert len(np.unique(np.round(u), axis=0)) == len(q)   # one point per voxel
        assert np.abs(q - np.clip(q, lo - 2 / (s * 512 * alpha), hi + 2 / (s * 512 * alpha))).max() == 0
    # two points in one voxel merge into one with the mean colour
    pts = np.array([[0, 0, 0], [1e-5, 0, 0], [1, 1, 1]], np.float32)
    cols = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    q, c = scenes.quantize_cloud(pts, cols)
    assert len(q) == 2
    np.testing.assert_allclose(c[np.argmin(q.sum(1))], [0.5, 0.5, 0.0])


def test_coarser_alpha_keeps_fewer_points_and_subsample_size():
    xyz, rgb, _, _ = scenes.humanoid_cloud(40_000, seed=1)
    counts = [len(scenes.quantize_cloud(xyz, rgb, alpha=a)[0]) for a in (1.0, 0.5, 0.25)]
    assert counts[0] >= counts[1] >= counts[2]
    s, c = scenes.subsample_cloud(xyz, rgb, 0.25, seed=3)
    assert len(s) == 10_000 and len(np.unique(s, axis=0)) == 10_000

"""Pins of the oracle's late shading (relighting from the normal map) and of
the global isotropic baseline's point spacing, against closed forms, a
library k-d tree and rotation invariance."""
import math

import numpy as np
import pytest

import oracle


def _px(v):
    """(3,) -> (3, 1, 1) single-pixel plane."""
    return np.asarray(v, np.float64).reshape(3, 1, 1)


def test_relight_lambert_closed_forms():
    rgb = _px([0.5, 0.25, 1.0])
    a = np.ones((1, 1))
    light = [(0.0, 0.0, 3.0, 0.8)]                # direction normalised by the shader
    cases = {(0, 0, 2): 1.0,                      # facing the light: ambient + I
             (0, 0, -1): 0.2,                     # facing away: ambient only
             (1, 0, 0): 0.2,                      # grazing: ambient only
             (0, math.sin(math.pi / 3), math.cos(math.pi / 3)): 0.2 + 0.8 * 0.5}
    for n, s in cases.items():
        out = oracle.relight(rgb, _px(n), a, light, 0.2)
        np.testing.assert_allclose(out, rgb * s, rtol=1e-15, atol=1e-15)
    # two lights add
    out = oracle.relight(rgb, _px((0, 0, 1)), a, light + [(0, 0, 1, 0.5)], 0.1)
    np.testing.assert_allclose(out, rgb * (0.1 + 0.8 + 0.5), rtol=1e-15)


def test_relight_no_normal_and_background():
    bg = (0.1, 0.2, 0.3)
    rgb = _px([0.7, 0.6, 0.5])
    # no normal (nothing rendered there): unshaded
    out = oracle.relight(rgb, _px((0, 0, 0)), np.full((1, 1), 0.4), [(0, 0, 1, 1.0)], 0.0, bg)
    np.testing.assert_allclose(out, rgb, rtol=1e-15)
    # pure background (alpha 0, rgb = bg): unchanged by any shading
    out = oracle.relight(_px(bg), _px((0, 0, 1)), np.zeros((1, 1)), [(0, 0, 1, 5.0)], 3.0, bg)
    np.testing.assert_allclose(out, _px(bg), rtol=1e-15)
    # the background part is not shaded: half coverage over a background
    C = np.array([0.2, 0.2, 0.2])
    rgb = _px(C + 0.5 * np.asarray(bg))
    out = oracle.relight(rgb, _px((0, 0, 1)), np.full((1, 1), 0.5), [(0, 0, 1, 1.0)], 0.5, bg)
    np.testing.assert_allclose(out, _px(1.5 * C + 0.5 * np.asarray(bg)), rtol=1e-14)


def test_relight_rotation_invariance():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(0)
    H, W = 5, 7
    rgb = rng.random((3, H, W))
    N = rng.standard_normal((3, H, W))
    a = rng.random((H, W))
    lights = [tuple(rng.standard_normal(3)) + (0.7,), tuple(rng.standard_normal(3)) + (0.4,)]
    R = Rot.random(random_state=3).as_matrix()
    Nr = np.einsum("ij,jhw->ihw", R, N)
    lr = [tuple(R @ np.array(l[:3])) + (l[3],) for l in lights]
    np.testing.assert_allclose(oracle.relight(rgb, N, a, lights, 0.15, (0.3, 0.1, 0.2)),
                               oracle.relight(rgb, Nr, a, lr, 0.15, (0.3, 0.1, 0.2)), rtol=1e-12, atol=1e-14)


def test_mean_nn_distance_grid_and_kdtree():
    # a regular grid of spacing 0.25 (exact in fp32): every nearest distance is 0.25
    g = np.stack(np.meshgrid(*[np.arange(6) * 0.25] * 3, indexing="ij"), -1).reshape(-1, 3)
    assert oracle.mean_nn_distance(g.astype(np.float32)) == 0.25
    kd = pytest.importorskip("scipy.spatial").cKDTree
    rng = np.random.default_rng(1)
    x = rng.random((3000, 3)).astype(np.float32)
    d, _ = kd(x.astype(np.float64)).query(x.astype(np.float64), k=2)
    np.testing.assert_allclose(oracle.mean_nn_distance(x), d[:, 1].mean(), rtol=1e-12)


def test_global_estimate_is_isotropic_at_the_mean_spacing():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2000, 3)).astype(np.float32)
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    c = rng.random((2000, 3)).astype(np.float32)
    e = oracle.estimate_global(x, c, 1.5, opacity=0.7)
    d = oracle.mean_nn_distance(x)
    np.testing.assert_allclose(e["scale"], np.float32(1.5 * d), rtol=0)
    assert (e["quat"] == np.array([1, 0, 0, 0], np.float32)).all()
    assert (e["opacity"] == np.float32(0.7)).all()
    # the normal is the kNN-PCA normal (on the unit sphere: nearly radial,
    # within the tilt of a 16-point patch of the curved surface)
    np.testing.assert_array_equal(e["normal"], oracle.pca(x, oracle.knn(x)[0])["normal"].astype(np.float32))
    assert np.abs(np.abs((e["normal"] * x).sum(1)) - 1).max() < 1e-2


# ------------------------------------------------------------ point raster
def _cam(W=5, H=4, f=10.0):
    return dict(viewmat=[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], fx=f, fy=f, cx=W / 2, cy=H / 2, width=W, height=H,
                near=0.01)


def test_point_raster_hand_example():
    cam = _cam()
    xyz = np.array([[0.0, 0.0, 1.0],     # u = 2.5, v = 2.0 -> pixel (2, 2)
                    [0.0, 0.0, 0.5],     # same pixel, nearer: wins
                    [0.0, 0.0, 0.5],     # same depth, higher index: loses
                    [0.0, 0.0, -1.0],    # behind the camera
                    [1.0, 0.0, 1.0],     # u = 12.5: outside
                    [-0.2, -0.15, 1.0]], np.float32)  # u = 0.5, v = 0.5 -> pixel (0, 0)
    rgb = np.arange(18, dtype=np.float32).reshape(6, 3) / 20
    r = oracle.point_raster(xyz, rgb, cam, bg=(0.5, 0.5, 0.5))
    assert r["winner"][2, 2] == 1 and r["winner"][0, 0] == 5
    assert (r["winner"] >= 0).sum() == 2
    np.testing.assert_array_equal(r["rgb"][:, 2, 2], rgb[1])
    np.testing.assert_array_equal(r["rgb"][:, 1, 1], [0.5, 0.5, 0.5])
    assert r["depth"][2, 2] == np.float32(0.5) and r["depth"][1, 1] == 0


def test_point_raster_matches_brute_force():
    rng = np.random.default_rng(4)
    cam = _cam(13, 9, 7.0)
    xyz = np.concatenate([rng.uniform(-1, 1, (400, 2)), rng.uniform(-0.5, 3, (400, 1))], 1).astype(np.float32)
    xyz[::7] = xyz[3]                         # duplicates: equal depths, ties by index
    rgb = rng.random((400, 3)).astype(np.float32)
    r = oracle.point_raster(xyz, rgb, cam)
    f32 = np.float32
    best = {}
    for i, (px, py, pz) in enumerate(xyz):
        x, y, z = f32(px), f32(py), f32(pz)       # identity camera: x, y, z exact
        if not (z > f32(0.01)):
            continue
        u = f32(7.0) * f32(x / z) + f32(6.5)
        v = f32(7.0) * f32(y / z) + f32(4.5)
        if not (0 <= u < 13 and 0 <= v < 9):
            continue
        key = (int(np.floor(v)), int(np.floor(u)))
        if key not in best or (z, i) < best[key]:
            best[key] = (z, i)
    w = np.full((9, 13), -1)
    for (j, i), (_, k) in best.items():
        w[j, i] = k
    np.testing.assert_array_equal(r["winner"], w)

"""Pins of the FP64 oracle renderer against closed forms, invariants, a
library rotation and an independent brute-force renderer (CPU only)."""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
import scenes
from brute_render import brute_render

CFG = oracle.DEFAULT_CFG


def ident_cam(W, H, f, near=0.01):
    v = np.zeros((3, 4), np.float32)
    v[:, :3] = np.eye(3)
    return dict(viewmat=v, fx=f, fy=f, cx=W / 2, cy=H / 2, width=W, height=H, near=near)


def one_gauss(mean, scale, quat=(1, 0, 0, 0), o=0.8, rgb=(0.9, 0.3, 0.1), nrm=(0, 0, -1)):
    return dict(mean=np.array([mean], np.float32), scale=np.array([scale], np.float32),
                quat=np.array([quat], np.float32), opacity=np.array([o], np.float32),
                rgb=np.array([rgb], np.float32), normal=np.array([nrm], np.float32))


# ---------------------------------------------------------------- P1 ----
@pytest.mark.parametrize("quat", [(1, 0, 0, 0), (0.3, -0.5, 0.7, 0.2), (0, 0, 0, 2.0)])
def test_p1_isotropic_closed_form(quat):
    """One isotropic Gaussian on the optical axis: Sigma_s = ((f sigma/z0)^2 +
    lowpass) I, so the image is bg + alpha (c - bg) inside r <= 3 s with
    alpha = min(0.99, o exp(-r^2 / 2 s^2)) wherever alpha >= 1/255."""
    W = H = 40
    f, z0, sig, o = 50.0, 2.0, 0.12, 0.8
    c = np.array([0.9, 0.3, 0.1])
    bg = (0.2, 0.4, 0.6)
    g = one_gauss((0, 0, z0), (sig, sig, sig), quat, o, c)
    cam = ident_cam(W, H, f)
    # the renderer sees the fp32 inputs, widened exactly
    sig, o, c = float(g["scale"][0, 0]), float(g["opacity"][0]), g["rgb"][0].astype(np.float64)
    r = oracle.render(g, cam, {**CFG, "bg": bg})
    s2 = (f * sig / z0) ** 2 + CFG["lowpass"]
    ii, jj = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    r2 = (ii - W / 2) ** 2 + (jj - H / 2) ** 2
    al = np.minimum(CFG["alpha_max"], o * np.exp(-r2 / (2 * s2)))
    on = (r2 <= 9 * s2) & (al >= CFG["alpha_floor"])
    al = np.where(on, al, 0.0)
    exp_rgb = np.asarray(bg)[:, None, None] + al * (c - np.asarray(bg))[:, None, None]
    ok = ~r["flag"]
    assert ok.sum() > W * H - 8
    np.testing.assert_allclose(r["rgb"][:, ok], exp_rgb[:, ok], atol=1e-12)
    np.testing.assert_allclose(r["alpha"][ok], al[ok], atol=1e-12)
    np.testing.assert_allclose(r["depth"][ok], (al * z0)[ok], atol=1e-12)
    np.testing.assert_allclose(r["normal"][2][ok], -al[ok], atol=1e-12)
    assert (r["ncontrib"][ok] == on[ok]).all()


# ---------------------------------------------------------------- P2 ----
def test_p2_offaxis_screen_covariance():
    """Isotropic Gaussian off axis: Sigma_s = sigma^2 J J^T + lowpass I with
    J from Eq. 4 (checks the -x f/z^2 terms) and u = f x / z + cx."""
    rng = np.random.default_rng(5)
    W = H = 256
    f = 200.0
    for _ in range(20):
        x, y, z = rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), rng.uniform(1.0, 3.0)
        sig = rng.uniform(0.005, 0.05)
        q = rng.standard_normal(4)
        g = one_gauss((x, y, z), (sig,) * 3, q)
        p = oracle.project(g, ident_cam(W, H, f))
        x, y, z = (float(np.float32(v)) for v in (x, y, z))
        sig = float(np.float32(sig))
        J = np.array([[f / z, 0, -x * f / z ** 2], [0, f / z, -y * f / z ** 2]])
        Ss = sig ** 2 * J @ J.T + CFG["lowpass"] * np.eye(2)
        if not p["vis"][0]:
            continue
        np.testing.assert_allclose(p["cov2"][0], [Ss[0, 0], Ss[0, 1], Ss[1, 1]], rtol=1e-12)
        np.testing.assert_allclose(p["uv"][0], [f * x / z + W / 2, f * y / z + H / 2], rtol=1e-13)
        inv = np.linalg.inv(Ss)
        np.testing.assert_allclose(p["conic"][0], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-10)


def test_p2_quaternion_convention():
    """q = 90 deg about z maps the x axis onto y, so Sigma = diag(s2^2, s1^2,
    s3^2) (columns of R are the principal axes) and on axis
    Sigma_s = (f/z)^2 diag(s2^2, s1^2) + lowpass."""
    f, z = 100.0, 2.0
    s = (0.01, 0.03, 0.02)
    h = math.sqrt(0.5)
    p = oracle.project(one_gauss((0, 0, z), s, (h, 0, 0, h)), ident_cam(128, 128, f))
    k = (f / z) ** 2
    s32 = np.float32(s).astype(np.float64)
    lp = CFG["lowpass"]
    np.testing.assert_allclose(p["cov2"][0], [k * s32[1] ** 2 + lp, 0.0, k * s32[0] ** 2 + lp],
                               rtol=1e-7, atol=1e-12)


def test_projection_vs_library_rotation():
    """Random anisotropic Gaussians under a random camera: the oracle's
    Sigma_s equals J T R S^2 R^T T^T J^T + lowpass I with R from scipy."""
    rng = np.random.default_rng(11)
    cam = scenes.look_at_camera((0.3, -0.2, -2.5), (0, 0, 0), (0, 1, 0), 50, 200, 150)
    n = 200
    g = dict(mean=rng.uniform(-0.5, 0.5, (n, 3)).astype(np.float32),
             scale=rng.uniform(0.001, 0.05, (n, 3)).astype(np.float32),
             quat=rng.standard_normal((n, 4)).astype(np.float32),
             opacity=np.ones(n, np.float32), rgb=np.ones((n, 3), np.float32),
             normal=np.ones((n, 3), np.float32))
    p = oracle.project(g, cam)
    V = cam["viewmat"].astype(np.float64)
    T, t = V[:, :3], V[:, 3]
    f = float(np.float32(cam["fx"]))
    for i in range(n):
        if not p["vis"][i]:
            continue
        x, y, z = T @ g["mean"][i].astype(np.float64) + t
        q = g["quat"][i].astype(np.float64)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        Sig = R @ np.diag(g["scale"][i].astype(np.float64) ** 2) @ R.T
        J = np.array([[f / z, 0, -x * f / z ** 2], [0, f / z, -y * f / z ** 2]])
        Ss = J @ T @ Sig @ T.T @ J.T + CFG["lowpass"] * np.eye(2)
        np.testing.assert_allclose(p["cov2"][i], [Ss[0, 0], Ss[0, 1], Ss[1, 1]],
                                   rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------- P3 ----
def _random_scene(seed, n, W, H):
    rng = np.random.default_rng(seed)
    cam = scenes.look_at_camera((0, 0, -2.0), (0, 0, 0), (0, 1, 0), 50, W, H)
    g = dict(mean=rng.uniform(-0.4, 0.4, (n, 3)).astype(np.float32),
             scale=rng.uniform(0.01, 0.08, (n, 3)).astype(np.float32),
             quat=rng.standard_normal((n, 4)).astype(np.float32),
             opacity=rng.uniform(0.2, 1.0, n).astype(np.float32),
             rgb=rng.random((n, 3)).astype(np.float32),
             normal=rng.standard_normal((n, 3)).astype(np.float32))
    return g, cam


def test_p3_zero_opacity_is_background():
    g, cam = _random_scene(1, 64, 48, 32)
    g["opacity"][:] = 0
    bg = (0.25, 0.5, 0.75)
    r = oracle.render(g, cam, {**CFG, "bg": bg})
    assert (r["rgb"] == np.asarray(bg)[:, None, None]).all()
    assert (r["normal"] == 0).all() and (r["depth"] == 0).all() and (r["alpha"] == 0).all()


def test_p3_weights_sum_and_cutoff():
    """With white colours and black background the colour is the weight sum
    sum_k alpha_k T_k, which must equal 1 - T_final, stay <= 1 - t_min and,
    since T only shrinks, be non-decreasing as Gaussians are added behind."""
    g, cam = _random_scene(2, 300, 64, 48)
    g["rgb"][:] = 1.0
    r = oracle.render(g, cam)
    np.testing.assert_allclose(r["rgb"][0], r["alpha"], atol=1e-12)
    assert r["alpha"].max() <= 1.0 - CFG["t_min"] + 1e-15
    assert r["alpha"].min() >= 0.0
    assert r["alpha"].max() > 0.99  # the scene does saturate somewhere
    # add one large opaque splat behind everything: coverage never decreases
    g2 = {k: np.concatenate([v, v[:1]]) for k, v in g.items()}
    g2["mean"][-1] = (0, 0, 1.5)
    g2["scale"][-1] = (0.6, 0.6, 0.01)
    g2["quat"][-1] = (1, 0, 0, 0)
    r2 = oracle.render(g2, cam)
    ok = ~(r["flag"] | r2["flag"])
    assert (r2["alpha"][ok] >= r["alpha"][ok] - 1e-15).all()


# ---------------------------------------------------------------- P4 ----
@pytest.mark.parametrize("seed,n,W,H", [(1, 1, 8, 8), (2, 3, 16, 8), (3, 8, 32, 32),
                                        (4, 8, 24, 16), (5, 40, 32, 24)])
def test_p4_brute_force_numpy(seed, n, W, H):
    g, cam = _random_scene(seed, n, W, H)
    bg = (0.1, 0.0, 0.3)
    r = oracle.render(g, cam, {**CFG, "bg": bg})
    rb = oracle.render(g, cam, {**CFG, "bg": bg}, brute=True)
    b = brute_render(g, cam, bg=bg)
    ok = ~r["flag"]
    for key in ("rgb", "normal"):
        np.testing.assert_array_equal(r[key], rb[key])
        np.testing.assert_allclose(r[key][:, ok], b[key][:, ok], atol=1e-10)
    for key in ("depth", "alpha"):
        np.testing.assert_allclose(r[key][ok], b[key][ok], atol=1e-10)


def test_row_lists_equal_literal_definition_cfg1():
    g = scenes.sphere_cloud()
    cam = scenes.look_at_camera((0, 0, -3), (0, 0, 0), (0, -1, 0), 60, 128, 128)
    r = oracle.render(g, cam)
    rb = oracle.render(g, cam, brute=True)
    for key in ("rgb", "normal", "depth", "alpha", "ncontrib", "last", "flag"):
        np.testing.assert_array_equal(r[key], rb[key])


# ---------------------------------------------------------------- P5 ----
def _rotation_quat(axis, ang):
    axis = np.asarray(axis, np.float64) / np.linalg.norm(axis)
    return np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])


def _qmul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b.T
    return np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)


def test_p5_permutation_invariance():
    g, cam = _random_scene(7, 200, 48, 40)
    perm = np.random.default_rng(0).permutation(200)
    gp = {k: v[perm] for k, v in g.items()}
    r, rp = oracle.render(g, cam), oracle.render(gp, cam)
    for key in ("rgb", "normal", "depth", "alpha", "ncontrib"):
        np.testing.assert_array_equal(r[key], rp[key])


def test_p5_corotation_invariance():
    """Rotating the world and the camera together leaves colour, depth and
    alpha unchanged and rotates the normal image."""
    g, cam = _random_scene(8, 150, 48, 40)
    ax, ang = np.array([0.3, 1.0, -0.2]), 0.7
    qQ = _rotation_quat(ax, ang)
    Q = Rotation.from_quat([*qQ[1:], qQ[0]]).as_matrix()
    g2 = dict(g)
    g2["mean"] = (g["mean"].astype(np.float64) @ Q.T).astype(np.float32)
    g2["quat"] = _qmul(qQ, g["quat"].astype(np.float64)).astype(np.float32)
    g2["normal"] = (g["normal"].astype(np.float64) @ Q.T).astype(np.float32)
    cam2 = dict(cam)
    v = cam["viewmat"].astype(np.float64)
    cam2["viewmat"] = np.concatenate([v[:, :3] @ Q.T, v[:, 3:]], 1).astype(np.float32)
    r, r2 = oracle.render(g, cam), oracle.render(g2, cam2)
    ok = ~(r["flag"] | r2["flag"])
    # inputs are re-rounded to fp32 after the rotation: allow that noise
    np.testing.assert_allclose(r2["rgb"][:, ok], r["rgb"][:, ok], atol=2e-5)
    np.testing.assert_allclose(r2["alpha"][ok], r["alpha"][ok], atol=2e-5)
    np.testing.assert_allclose(r2["depth"][ok], r["depth"][ok], atol=5e-5)
    nrot = np.einsum("ij,jhw->ihw", Q, r["normal"])
    np.testing.assert_allclose(r2["normal"][:, ok], nrot[:, ok], atol=5e-5)


# ---------------------------------------------------------------- binning
def test_binning_hand_derived_2x2():
    """On-axis Gaussian at the centre of a 64x64 image, screen sigma 2 px
    (lowpass 0): the box is x,y in [26, 37], i.e. tiles 1..2 in x and y of
    a 4x4 grid -> ids 5, 6, 9, 10, each keyed with the fp32 depth bits."""
    f, z = 100.0, 2.5
    sig = 2.0 * z / f
    g = one_gauss((0, 0, z), (sig,) * 3)
    cam = ident_cam(64, 64, f)
    cfg = {**CFG, "lowpass": 0.0}
    p = oracle.project(g, cam, cfg)
    assert list(p["prect"][0]) == [26, 37, 26, 37]
    keys, vals, ranges = oracle.bin_keys([p], [cam], cfg)
    zb = int(np.float32(z).view(np.uint32))
    assert [int(k) for k in keys] == [(t << 32) | zb for t in (5, 6, 9, 10)]
    assert (vals == 0).all()
    assert ranges[5].tolist() == [0, 1] and ranges[10].tolist() == [3, 4]
    assert ranges[0].tolist() == [0, 0]


def test_binning_structure_and_tile_invariance():
    """For tile sizes 8/16/32: K = sum of per-Gaussian tile counts, keys
    ascend, equal keys keep ascending Gaussian index, every contributing
    (pixel, Gaussian) pair of the image lies in that pixel's tile list, and
    the image itself does not depend on the tile size."""
    g, cam = _random_scene(9, 400, 80, 48)
    imgs = []
    for B in (8, 16, 32):
        cfg = {**CFG, "tile": B}
        p = oracle.project(g, cam, cfg)
        keys, vals, ranges = oracle.bin_keys([p], [cam], cfg)
        assert len(keys) == int(p["ntiles"].sum())
        assert (np.diff(keys.astype(np.uint64)) >= 0).all()
        same = keys[1:] == keys[:-1]
        assert (vals[1:][same] > vals[:-1][same]).all()
        r = oracle.render(g, cam, cfg, proj=p)
        imgs.append(r["rgb"])
        tx = -(-cam["width"] // B)
        # each pixel's last contributor is in the pixel's tile list
        for j in range(0, cam["height"], 3):
            for i in range(0, cam["width"], 3):
                gl = r["last"][j, i]
                if gl < 0:
                    continue
                t = (j // B) * tx + i // B
                s, e = ranges[t]
                assert gl in set(vals[s:e].tolist())
    np.testing.assert_array_equal(imgs[0], imgs[1])
    np.testing.assert_array_equal(imgs[0], imgs[2])


def test_near_plane_and_zero_quaternion_cull():
    g = one_gauss((0, 0, 0.005), (0.01,) * 3)
    p = oracle.project(g, ident_cam(32, 32, 50.0))
    assert p["vis"][0] == 0 and p["ntiles"][0] == 0
    g = one_gauss((0, 0, 2.0), (0.01,) * 3, (0, 0, 0, 0))
    p = oracle.project(g, ident_cam(32, 32, 50.0))
    assert p["vis"][0] == 0

"""Pin of the ground-truth ray caster: a sphere's closed-form silhouette,
centre depth and normal, and a capped cylinder seen end-on (its disk)."""
import math

import numpy as np

import oracle
import scenes


def test_sphere_closed_form():
    r, D, W = 0.3, 2.0, 128
    prim = scenes.Primitive("ell", center=np.zeros(3), radii=np.full(3, r))
    cam = scenes.look_at_camera((0, 0, -D), (0, 0, 0), (0, -1, 0), 40, W, W)
    g = oracle.raycast([prim], cam)
    f = cam["fx"]
    rad_px = f * r / math.sqrt(D * D - r * r)          # silhouette radius
    ii, jj = np.meshgrid(np.arange(W) + 0.5, np.arange(W) + 0.5)
    rr = np.hypot(ii - W / 2, jj - W / 2)
    clear = np.abs(rr - rad_px) > 0.02
    assert (g["hit"][clear] == (rr < rad_px)[clear]).all()
    c = W // 2
    np.testing.assert_allclose(g["depth"][c, c], D - r, atol=1e-3)   # pixel centre is 0.5 px off axis
    np.testing.assert_allclose(g["normal"][:, c, c], [0, 0, -1], atol=2e-2)
    # every hit is on the sphere with a radial unit normal
    P = g["point"][g["hit"]]
    np.testing.assert_allclose(np.linalg.norm(P, axis=1), r, rtol=1e-12)
    np.testing.assert_allclose(g["normal"][:, g["hit"]].T, P / r, atol=1e-12)


def test_capped_cylinder_end_on_is_a_disk():
    prim = scenes.Primitive("cyl", p0=np.array([0, 0, 0.5]), p1=np.array([0, 0, -0.5]), r=0.2)
    D, W = 3.0, 96
    cam = scenes.look_at_camera((0, 0, -D), (0, 0, 0), (0, -1, 0), 30, W, W)
    g = oracle.raycast([prim], cam)
    f = cam["fx"]
    rad_px = f * 0.2 / (D - 0.5)                       # the near cap at depth D - 0.5
    ii, jj = np.meshgrid(np.arange(W) + 0.5, np.arange(W) + 0.5)
    rr = np.hypot(ii - W / 2, jj - W / 2)
    clear = np.abs(rr - rad_px) > 0.02
    assert (g["hit"][clear] == (rr < rad_px)[clear]).all()
    np.testing.assert_allclose(g["depth"][g["hit"]], D - 0.5, rtol=1e-12)
    np.testing.assert_allclose(g["normal"][2][g["hit"]], -1.0)


def test_scene_gt_views_match_oracle_raycast():
    """The training targets (scenes.gt_views, numpy) equal the oracle's
    exact C ray caster on the humanoid proxy."""
    prims = scenes.humanoid_primitives()
    cam = scenes.sphere_camera(np.array([0, 0.5, 0]), 2.5, np.random.default_rng(3), 192, 160)
    g = scenes.gt_views(prims, [cam])[0]
    o = oracle.raycast(prims, cam, texture=scenes.texture)
    assert (g["hit"] == o["hit"]).all() and o["hit"].sum() > 200
    np.testing.assert_allclose(g["depth"], o["depth"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(g["normal"], o["normal"], atol=1e-9)
    np.testing.assert_allclose(g["rgb"], o["rgb"], atol=1e-9)

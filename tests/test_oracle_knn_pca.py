"""Pins of the kNN-PCA oracle: brute force and a library k-d tree for the
neighbours, numpy for covariance and eigen-decomposition, scipy for the
quaternion, closed forms on planes and lines."""
import numpy as np
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

import oracle
import scenes


def test_knn_brute_force_with_index_ties():
    rng = np.random.default_rng(0)
    # integer grid points: many exact distance ties
    p = rng.integers(0, 6, (400, 3)).astype(np.float32) * 0.01
    p = np.unique(p, axis=0)
    idx, d2 = oracle.knn(p)
    P = p.astype(np.float64)
    D = ((P[:, None, :] - P[None, :, :]) ** 2).sum(-1)
    for i in range(len(p)):
        order = np.lexsort((np.arange(len(p)), D[i]))
        order = order[order != i][:16]
        assert list(idx[i]) == list(order)
        np.testing.assert_array_equal(d2[i], D[i, order])


def test_knn_distances_match_kdtree():
    xyz, _, _, _ = scenes.humanoid_cloud(20_000, seed=4)
    idx, d2 = oracle.knn(xyz)
    dd, _ = cKDTree(xyz.astype(np.float64)).query(xyz.astype(np.float64), k=17)
    np.testing.assert_allclose(np.sqrt(d2), dd[:, 1:], rtol=1e-12, atol=1e-15)


def test_pca_plane_line_and_numpy():
    rng = np.random.default_rng(1)
    # points on a tilted plane: the normal is the plane normal, l3 = 0
    u, v = np.meshgrid(np.arange(30), np.arange(30))
    nrm = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    a = np.cross(nrm, [1, 0, 0]); a /= np.linalg.norm(a)
    b = np.cross(nrm, a)
    pts = (0.01 * u.reshape(-1, 1) * a + 0.01 * v.reshape(-1, 1) * b + 0.3).astype(np.float32)
    idx, _ = oracle.knn(pts)
    e = oracle.pca(pts, idx)
    assert np.abs(np.abs(e["normal"] @ nrm) - 1).max() < 1e-5
    assert (np.abs(e["lam"][:, 2]) < 1e-10 * e["lam"][:, 0] + 1e-14).all()
    # against numpy: covariance (biased, over the neighbours) and eigenvalues
    p = rng.standard_normal((3000, 3)).astype(np.float32) * np.float32([0.05, 0.02, 0.01])
    idx, _ = oracle.knn(p)
    e = oracle.pca(p, idx)
    for i in rng.choice(3000, 50, replace=False):
        Nb = p[idx[i]].astype(np.float64)
        C = np.cov(Nb.T, bias=True)
        cv = e["cov"][i]
        np.testing.assert_allclose([cv[0], cv[1], cv[2], cv[3], cv[4], cv[5]],
                                   [C[0, 0], C[0, 1], C[0, 2], C[1, 1], C[1, 2], C[2, 2]], rtol=1e-10,
                                   atol=1e-16)
        w = np.linalg.eigvalsh(C)[::-1]
        np.testing.assert_allclose(e["lam"][i], w, rtol=1e-9, atol=1e-15)
        # quaternion: proper rotation whose columns are the axes; Sigma rebuilt
        R = Rotation.from_quat([*e["quat"][i][1:], e["quat"][i][0]]).as_matrix()
        assert np.linalg.det(R) > 0
        np.testing.assert_allclose(R[:, 2], e["normal"][i], atol=1e-9)
        s = e["scale"][i]
        if s[2] > 0.1 * s[1] * (1 + 1e-12):   # unclamped: Sigma == kappa^2 Cov
            np.testing.assert_allclose(R @ np.diag(s ** 2) @ R.T, C, rtol=1e-7, atol=1e-14)


def test_pca_normals_point_outwards_on_sphere():
    g = scenes.sphere_cloud(5000, seed=2)
    idx, _ = oracle.knn(g["mean"])
    e = oracle.pca(g["mean"], idx)
    cos = (e["normal"] * g["mean"]).sum(1)
    assert (cos > 0.95).all()

"""The oracle against hand-derived worked examples stored under tests/golden/.

Each fixture states its inputs (exact binary fractions, so the expected
values are exact), the passage of the paper it works through and the
derivation by hand; the values were not produced by any program.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    """Non-comment lines of a fixture, split into words."""
    out = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if line:
                out.append(line)
    return out


def _num(s):
    return float(Fraction(s))


def _camera(words):
    kv = dict(zip(words[1::2], words[2::2]))
    W, H = int(kv["width"]), int(kv["height"])
    v = np.zeros((3, 4), np.float32)
    v[:, :3] = np.eye(3)
    return dict(viewmat=v, fx=_num(kv["fx"]), fy=_num(kv["fy"]), cx=_num(kv["cx"]), cy=_num(kv["cy"]),
                width=W, height=H, near=0.01)


def test_eq1_stacked_splats():
    """Sec. 3.1, Eq. 1-2: three splats on one pixel, composited by depth."""
    rows = _rows("eq1_stacked_splats.txt")
    sp = np.array([[_num(x) for x in r[1:]] for r in rows if r[0] == "splat"])
    cam = _camera(next(r for r in rows if r[0] == "camera"))
    exp = {r[0]: [_num(x) for x in r[1:]] for r in rows if r[0] not in ("splat", "camera")}
    g = dict(mean=sp[:, 0:3], scale=sp[:, 3:6], quat=sp[:, 6:10], opacity=sp[:, 10],
             rgb=sp[:, 11:14], normal=sp[:, 14:17])
    g = {k: np.ascontiguousarray(v, np.float32) for k, v in g.items()}
    # the inputs are exact in fp32, so the derivation holds for the widened values
    assert all((g[k].astype(np.float64) == v).all() for k, v in
               dict(mean=sp[:, 0:3], opacity=sp[:, 10], rgb=sp[:, 11:14]).items())
    px, py = (int(v) for v in exp["pixel"])
    for brute in (False, True):
        r = oracle.render(g, cam, {**oracle.DEFAULT_CFG, "bg": (0.0, 0.0, 0.0)}, brute=brute)
        assert not r["flag"][py, px]
        np.testing.assert_allclose(r["rgb"][:, py, px], exp["rgb"], rtol=0, atol=1e-15)
        assert r["depth"][py, px] == pytest.approx(exp["depth"][0], abs=1e-15)
        assert r["alpha"][py, px] == pytest.approx(exp["alpha"][0], abs=1e-15)
        np.testing.assert_allclose(r["normal"][:, py, px], exp["normal"], rtol=0, atol=1e-15)
        assert int(r["last"][py, px]) == int(exp["last"][0])
        assert int(r["ncontrib"][py, px]) == int(exp["ncontrib"][0])


@pytest.mark.parametrize("case", ["axis", "turned"])
def test_eq3_projected_covariance(case):
    """Sec. 3.1, Eq. 3-4: screen covariance, its conic and the screen mean."""
    rows = _rows("eq3_projected_covariance.txt")
    cam = _camera(next(r for r in rows if r[0] == "camera"))
    gw = [_num(x) for x in next(r for r in rows if r[0] == "gaussian")[1:]]
    row = next(r for r in rows if r[0] == "case" and r[1] == case)
    q = [_num(x) for x in row[2:6]]
    cov = [_num(x) for x in row[6:9]]
    conic = [_num(x) for x in row[9:12]]
    uv = [_num(x) for x in next(r for r in rows if r[0] == "uv")[1:]]
    g = dict(mean=np.array([gw[0:3]], np.float32), scale=np.array([gw[3:6]], np.float32),
             quat=np.array([q], np.float32))
    p = oracle.project(g, cam, {**oracle.DEFAULT_CFG, "lowpass": 0.0})
    assert p["vis"][0]
    np.testing.assert_allclose(p["cov2"][0], cov, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(p["conic"][0], conic, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(p["uv"][0], uv, rtol=0, atol=1e-12)
    assert p["xyz"][0].tolist() == gw[0:3]


def test_knn_pca_square_grid():
    """Sec. 2.1 prior (k = 16 kNN-PCA): a query amid 16 plane points at four
    distances, ties in index order, covariance diag(1.875, 1.875, 0)."""
    rows = _rows("knn_pca_square_grid.txt")
    pts = sorted((int(r[1]), [_num(x) for x in r[2:5]]) for r in rows if r[0] == "point")
    xyz = np.array([p for _, p in pts], np.float32)
    exp = {r[0]: [_num(x) for x in r[1:]] for r in rows if r[0] != "point"}
    q = int(exp["query"][0])
    idx, d2 = oracle.knn(xyz)
    assert idx[q].tolist() == [int(v) for v in exp["neighbours"]]
    assert d2[q].tolist() == exp["d2"]
    e = oracle.pca(xyz, idx)
    np.testing.assert_allclose(e["lam"][q], exp["lambda"], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(e["scale"][q], exp["scale"], rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(e["normal"][q], exp["normal"], atol=1e-14)

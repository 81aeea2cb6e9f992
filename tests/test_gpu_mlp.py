"""Learned estimator on tcgen05 (p2e_estimate mode 1) against the oracle's
FP64 network on bf16-rounded operands (R10).

Tolerance: 1e-2 relative on every output element (the element-wise
maximum), over the well-conditioned points.  Bit agreement is not
expected: the accumulation order differs, and a feature or activation can
round to a neighbouring bf16 value when fp32 and fp64 straddle a rounding
boundary.  A point is excluded (counted, the count bounded) when one of
the discrete decisions that shape its features is taken at a knife edge,
where fp32 and fp64 may legitimately disagree:
  * its 16 neighbours come in a different order (two neighbour distances
    equal in fp32 but not in fp64: the features are permuted);
  * two PCA eigenvalues within 1e-3 of the largest (the frame is
    ill-conditioned);
  * the canonical frame's sign choices are ambiguous: the first axis's
    two largest components within 1e-3 of each other in magnitude, or the
    point within 1e-4 m of the plane through the centroid normal to its
    axis (the normal's orientation).
The 800K-point case runs the kernel's multi-tile loop: 6250 tiles of 128
points over a persistent grid of at most three CTAs per SM, about 14
tiles per CTA, so the next-tile prefetch, the reuse of the shared A/H
buffers and the mbarrier phase across tiles are all exercised.
"""
import numpy as np
import pytest
import torch

import oracle.mlp as om
import scenes

pytestmark = pytest.mark.gpu


def _params(seed, scale_out=0.3):
    from paper_2409_16504_gb300 import mlp
    p = mlp.init_params(seed, device="cpu")
    g = torch.Generator().manual_seed(seed + 1)
    p["W4"] = torch.randn((mlp.OUT_PAD, mlp.HID), generator=g) * scale_out / 8
    p["W4"][mlp.OUT:] = 0
    for k in mlp.BIASES:
        p[k] = torch.randn(mlp.SHAPES[k], generator=g) * 0.05
    p["b4"][mlp.OUT:] = 0
    return p


def _gpu(xyz, rgb, p, mode=1):
    from paper_2409_16504_gb300 import mlp
    from paper_2409_16504_gb300.estimate import Estimator, cloud_tensors
    a, b = cloud_tensors(xyz, rgb)
    n = len(xyz)
    blob = mlp.pack({k: v.cuda() for k, v in p.items()})
    knn = torch.zeros((n, 16), dtype=torch.int32, device="cuda")
    est = Estimator(n)
    gs = est(a, b, mode=mode, mlp_blob=blob, knn=knn)
    est.check(n)  # raises if a bounded device wait gave up
    out = {k: getattr(gs, k).cpu().numpy().astype(np.float64) for k in ("mean_op", "scale", "quat", "normal")}
    out["idx"] = knn.cpu().numpy().astype(np.int64)
    return out


def _well_conditioned(xyz, ref, got):
    lam = ref["pca"]["lam"]
    gaps = ((lam[:, 0] - lam[:, 1]) > 1e-3 * lam[:, 0]) & ((lam[:, 1] - lam[:, 2]) > 1e-3 * lam[:, 0])
    same_order = (got["idx"] == ref["idx"]).all(1)
    R = om.quat_to_rot(ref["pca"]["quat"])
    e0 = np.sort(np.abs(R[:, :, 0]), 1)
    axis_clear = (e0[:, 2] - e0[:, 1]) > 1e-3
    P = np.asarray(xyz, np.float64)
    side = ((P - P.mean(0)) * ref["pca"]["normal"]).sum(1)
    side_clear = np.abs(side) > 1e-4
    ok = gaps & same_order & axis_clear & side_clear
    print(f"excluded: order {int((~same_order).sum())}, eigen gap {int((~gaps).sum())}, "
          f"axis sign {int((~axis_clear).sum())}, normal side {int((~side_clear).sum())}; "
          f"kept {int(ok.sum())} of {len(ok)}")
    return ok


@pytest.mark.parametrize("n,seed", [(800_000, 2), (20_000, 5), (4096, 6)])
def test_mlp_matches_oracle(n, seed):
    xyz, rgb, _, _ = scenes.humanoid_cloud(n, seed=seed)
    p = _params(seed)
    got = _gpu(xyz, rgb, p)
    ref = om.estimate(xyz, rgb, {k: v.double().numpy() for k, v in p.items()})
    ok = _well_conditioned(xyz, ref, got)
    assert ok.mean() > 0.99
    # the corrections are not trivial
    assert np.abs(ref["y"][ok]).max() > 0.05
    rs = np.abs(got["scale"][ok, :3] - ref["scale"][ok]) / ref["scale"][ok]
    qd = np.abs((got["quat"][ok] * ref["quat"][ok]).sum(1) /
                np.linalg.norm(got["quat"][ok], axis=1) / np.linalg.norm(ref["quat"][ok], axis=1))
    ro = np.abs(got["mean_op"][ok, 3] - ref["opacity"][ok]) / ref["opacity"][ok]
    cn = (got["normal"][ok, :3] * ref["normal"][ok]).sum(1)
    print(f"max: scale rel {rs.max():.2e}, 1-|cos q| {(1 - qd).max():.2e}, opacity rel {ro.max():.2e}, "
          f"1-cos n {(1 - cn).max():.2e}")
    assert rs.max() < 1e-2
    assert (1 - qd).max() < 1e-3
    assert ro.max() < 1e-2
    assert (1 - cn).max() < 1e-3
    np.testing.assert_array_equal(got["mean_op"][:, :3], np.asarray(xyz, np.float32))


def test_zero_last_layer_reproduces_pca():
    from paper_2409_16504_gb300 import mlp
    xyz, rgb, _, _ = scenes.humanoid_cloud(8192, seed=7)
    p = mlp.init_params(1, device="cpu")
    a = _gpu(xyz, rgb, p, mode=1)
    b = _gpu(xyz, rgb, p, mode=0)
    np.testing.assert_array_equal(a["scale"], b["scale"])
    np.testing.assert_allclose(a["quat"], b["quat"], atol=1e-6)
    np.testing.assert_allclose(a["mean_op"], b["mean_op"], atol=1e-6)
    np.testing.assert_allclose(a["normal"], b["normal"], atol=1e-6)

"""Pins of the oracle's learned-estimator forward (oracle/mlp.py) against
facts fixed outside it: bf16 rounding against torch's conversion and the
round-half-to-even rule; the features of a hand-built neighbourhood in a
known frame; a selector network whose output is known in closed form; and
the output mapping's special cases (zero output = the PCA estimate, scale
doubling and clipping, an in-plane rotation increment composed on the right,
the opacity logit shift) against scipy's rotations."""
import math

import numpy as np
import pytest
import torch

import oracle.mlp as om


def test_bf16_round_half_even_and_torch():
    one = 1.0
    # bf16 spacing at 1 is 2^-7: 1 + 2^-8 ties down to 1 (even), 1 + 3 2^-8 ties up
    assert om.bf16_round(one + 2.0 ** -8) == 1.0
    assert om.bf16_round(one + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert om.bf16_round(one + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000), [0.0, -0.0, 1e-40]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(om.bf16_round(x), ref)


def test_features_of_a_hand_built_neighbourhood():
    """Point at (1, 2, 3), 16 neighbours at known offsets, frame = 90 degrees
    about z, so R^T d = (d_y, -d_x, d_z); r = |d_16|."""
    rng = np.random.default_rng(1)
    p0 = np.array([1.0, 2.0, 3.0])
    d = rng.standard_normal((16, 3))
    d *= (np.arange(1, 17) / np.linalg.norm(d, axis=1))[:, None]   # distances 1..16
    xyz = np.vstack([p0, p0 + d])
    rgb = rng.random((17, 3))
    idx = np.arange(1, 17)[None, :]
    c, s = math.cos(math.pi / 4), math.sin(math.pi / 4)
    idx_all = np.vstack([idx, np.zeros((16, 16), int)])      # rows 1..16 unused
    quat = np.vstack([[c, 0, 0, s], np.tile([1.0, 0, 0, 0], (16, 1))])
    f = om.features(xyz, rgb, idx_all, quat)[0]
    r = 16.0
    for k in range(16):
        dk = d[k]
        np.testing.assert_allclose(f[6 * k: 6 * k + 3], [dk[1] / r, -dk[0] / r, dk[2] / r], atol=1e-14)
        np.testing.assert_allclose(f[6 * k + 3: 6 * k + 6], rgb[k + 1] - rgb[0], atol=1e-15)


def _selector(perm, bias1=0.0):
    p = {k: np.zeros(shp) for k, shp in om.BF16_SHAPES + om.F32_SHAPES}
    for i in range(om.HID):
        p["W1"][i, perm[i]] = 1.0
    p["W2"][:] = np.eye(om.HID)
    p["W3"][:] = np.eye(om.HID)
    for i in range(om.OUT):
        p["W4"][i, i] = 1.0
    p["b1"][:] = bias1
    return p


def test_forward_selector_network_closed_form():
    rng = np.random.default_rng(2)
    x = rng.integers(-16, 17, (50, om.IN)) / 8.0           # exact in bf16
    perm = np.arange(om.IN - 1, om.IN - 1 - om.HID, -1)     # hidden i <- feature 95 - i
    y = om.forward(_selector(perm), x)
    np.testing.assert_array_equal(y, np.maximum(x[:, perm[:om.OUT]], 0.0))
    y2 = om.forward(_selector(perm, bias1=-0.5), x)
    np.testing.assert_array_equal(y2, np.maximum(x[:, perm[:om.OUT]] - 0.5, 0.0))
    # the bias of the last layer is added after the last matmul, without ReLU
    p = _selector(perm)
    p["b4"][:om.OUT] = -3.0
    np.testing.assert_array_equal(om.forward(p, x), np.maximum(x[:, perm[:om.OUT]], 0.0) - 3.0)


def test_output_mapping_special_cases():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(3)
    n = 6
    q0 = rng.standard_normal((n, 4))
    s0 = rng.uniform(0.01, 0.1, (n, 3))
    o0 = np.full(n, 0.9)
    base = Rot.from_quat(q0[:, [1, 2, 3, 0]])              # scipy is scalar-last
    R0 = base.as_matrix()
    # zero output: the PCA estimate itself
    out = om.apply_corrections(s0, q0, o0, np.zeros((n, 8)))
    np.testing.assert_allclose(out["scale"], s0, rtol=1e-15)
    np.testing.assert_allclose(out["quat"], q0 / np.linalg.norm(q0, axis=1, keepdims=True), atol=1e-15)
    np.testing.assert_allclose(out["opacity"], 0.9, rtol=1e-14)
    np.testing.assert_allclose(out["normal"], R0[:, :, 2], atol=1e-14)
    # scale: exp of the first three outputs, clipped at +-4
    y = np.zeros((n, 8))
    y[:, 0], y[:, 1], y[:, 2] = math.log(2.0), 10.0, -10.0
    out = om.apply_corrections(s0, q0, o0, y)
    np.testing.assert_allclose(out["scale"], s0 * [2.0, math.exp(4.0), math.exp(-4.0)], rtol=1e-14)
    # rotation increment (1, 0, 0, tan(theta/2)) = theta about the local normal:
    # R = R_pca Rz(theta); the normal is unchanged, e1 turns towards e2
    th = 0.7
    y = np.zeros((n, 8))
    y[:, 6] = math.tan(th / 2)
    out = om.apply_corrections(s0, q0, o0, y)
    Rn = om.quat_to_rot(out["quat"])
    np.testing.assert_allclose(Rn, (base * Rot.from_euler("z", th)).as_matrix(), atol=1e-14)
    np.testing.assert_allclose(out["normal"], R0[:, :, 2], atol=1e-14)
    np.testing.assert_allclose(Rn[:, :, 0], math.cos(th) * R0[:, :, 0] + math.sin(th) * R0[:, :, 1], atol=1e-14)
    # opacity: a logit shift
    y = np.zeros((n, 8))
    y[:, 7] = -math.log(0.9 / 0.1)
    np.testing.assert_allclose(om.apply_corrections(s0, q0, o0, y)["opacity"], 0.5, rtol=1e-14)

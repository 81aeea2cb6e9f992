"""p2e_loss_ssim (the SSIM term of an "L1 + SSIM" image loss) against the
FP64 oracle (oracle/ssim.py, itself pinned to scipy's Gaussian filter, a
closed form and central differences): the loss within 1e-5 relative and
the gradient element by element within 2e-3 of its largest entry (fp32
window sums and ratios), on two views of ragged sizes; the call
accumulates into the loss and the gradient buffers it is given."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle.ssim as os_

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sizes", [[(37, 29), (64, 48)], [(300, 200), (129, 517), (5, 3)]])
def test_ssim_loss_and_gradient_match_oracle(sizes):
    """Views smaller than, equal to and spanning many 32 x 16 tiles with
    ragged edges (and one smaller than the window)."""
    from paper_2409_16504_gb300 import _lib
    from paper_2409_16504_gb300.render import _ptr, _stream
    rng = np.random.default_rng(4)
    xs = [rng.random((3, h, w)).astype(np.float32) for h, w in sizes]
    ys = [np.clip(x + 0.15 * rng.standard_normal(x.shape), 0, 1).astype(np.float32) for x in xs]
    npix = sum(h * w for h, w in sizes)
    x_d = torch.from_numpy(np.concatenate([x.reshape(-1) for x in xs])).cuda()
    y_d = torch.from_numpy(np.concatenate([y.reshape(-1) for y in ys])).cuda()
    g0 = rng.standard_normal(3 * npix).astype(np.float32) * 1e-4
    d_rgb = torch.from_numpy(g0.copy()).cuda()
    loss = torch.full((1,), 0.5, device="cuda")
    scratch = torch.empty(96 * npix + 256, dtype=torch.uint8, device="cuda")
    sp = C.c_void_p((scratch.data_ptr() + 255) & ~255)
    hw = (C.c_int32 * (2 * len(sizes)))(*[v for h, w in sizes for v in (h, w)])
    w = 0.7
    st = _lib.load().p2e_loss_ssim(_ptr(x_d), _ptr(y_d), hw, len(sizes), C.c_float(w), _ptr(loss), _ptr(d_rgb), sp,
                                   96 * npix, _stream())
    assert st == 0
    torch.cuda.synchronize()
    D, g = os_.loss_and_grad([x.astype(np.float64) for x in xs], [y.astype(np.float64) for y in ys])
    np.testing.assert_allclose(loss.item(), 0.5 + w * D, rtol=1e-5)
    ref = w * np.concatenate([a.reshape(-1) for a in g])
    got = d_rgb.cpu().numpy().astype(np.float64) - g0.astype(np.float64)
    err = np.abs(got - ref).max() / np.abs(ref).max()
    print(f"SSIM term D = {D:.6f}; gradient max error {err:.2e} of its largest entry")
    assert err <= 2e-3


def test_ssim_rejects_bad_arguments():
    from paper_2409_16504_gb300 import _lib
    lib = _lib.load()
    t = torch.zeros(64, device="cuda")
    s = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    hw = (C.c_int32 * 2)(4, 4)
    p = C.c_void_p(t.data_ptr())
    sp = C.c_void_p((s.data_ptr() + 255) & ~255)
    assert lib.p2e_loss_ssim(p, p, hw, 1, C.c_float(1.0), p, p, sp, 16, None) == _lib.P2E_ERR_INVALID_ARG
    assert lib.p2e_loss_ssim(p, p, hw, 0, C.c_float(1.0), p, p, sp, 2048, None) == _lib.P2E_ERR_INVALID_ARG


def test_ssim_loss_sum_at_full_size():
    """The differentiation's shape, 8 views at 512^2 (6.3M window sums):
    the loss is the fp64 sum of the per-pixel fp32 S, added once, so it
    stays within 2e-6 of the FP64 value (per-block float atomics would
    round 12,288 times into the loss)."""
    from paper_2409_16504_gb300 import _lib
    from paper_2409_16504_gb300.render import _ptr, _stream
    rng = np.random.default_rng(8)
    sizes = [(512, 512)] * 8
    xs = [rng.random((3, h, w)).astype(np.float32) for h, w in sizes]
    ys = [np.clip(x + 0.1 * rng.standard_normal(x.shape), 0, 1).astype(np.float32) for x in xs]
    npix = sum(h * w for h, w in sizes)
    x_d = torch.from_numpy(np.concatenate([x.reshape(-1) for x in xs])).cuda()
    y_d = torch.from_numpy(np.concatenate([y.reshape(-1) for y in ys])).cuda()
    d_rgb = torch.zeros(3 * npix, device="cuda")
    loss = torch.zeros(1, device="cuda")
    scratch = torch.empty(96 * npix + 256, dtype=torch.uint8, device="cuda")
    sp = C.c_void_p((scratch.data_ptr() + 255) & ~255)
    hw = (C.c_int32 * (2 * len(sizes)))(*[v for h, w in sizes for v in (h, w)])
    assert _lib.load().p2e_loss_ssim(_ptr(x_d), _ptr(y_d), hw, len(sizes), C.c_float(1.0), _ptr(loss),
                                     _ptr(d_rgb), sp, 96 * npix, _stream()) == 0
    torch.cuda.synchronize()
    D = np.mean([os_.ssim_terms(x[c].astype(np.float64), y[c].astype(np.float64))["S"].mean()
                 for x, y in zip(xs, ys) for c in range(3)])
    assert abs(loss.item() - (1.0 - D)) <= 2e-6, (loss.item(), 1.0 - D)

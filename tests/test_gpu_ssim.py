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


def test_ssim_loss_and_gradient_match_oracle():
    from paper_2409_16504_gb300 import _lib
    from paper_2409_16504_gb300.render import _ptr, _stream
    rng = np.random.default_rng(4)
    sizes = [(37, 29), (64, 48)]
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
    hw = (C.c_int32 * 4)(sizes[0][0], sizes[0][1], sizes[1][0], sizes[1][1])
    w = 0.7
    st = _lib.load().p2e_loss_ssim(_ptr(x_d), _ptr(y_d), hw, 2, C.c_float(w), _ptr(loss), _ptr(d_rgb), sp,
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

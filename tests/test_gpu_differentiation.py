"""Differentiation at scale: a 200K-point humanoid, a batch of 8 views at
512^2, loss = Eq. 5 + 0.2 x the SSIM term against the exact ray-cast views,
forward and hand-written backward through every Gaussian parameter.  The
gradients' correctness is pinned on small scenes (tests/test_gpu_backward.py
against the FP64 oracle gradient, itself pinned to central differences);
here the full-scale run must complete, stay finite and descend: a step
against the gradient of the colours lowers the loss."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_differentiation_200k_8x512():
    from paper_2409_16504_gb300.render import p2e_render_backward
    from paper_2409_16504_gb300.train import Scene, Trainer, time_differentiation
    t = time_differentiation(points=200_000, views=8, res=512, ssim_weight=0.2, reps=2)
    print("differentiation 200K x 8 x 512^2:", {k: (round(v, 3) if isinstance(v, float) else v) for k, v in t.items()})
    assert t["gradients_finite"] and np.isfinite(t["loss"])
    assert t["keys"] > 200_000
    # a small step of the colours against their gradient lowers the loss
    sc = Scene(3, 200_000, 8, 512)
    tr = Trainer(200_000, ssim_weight=0.2)
    _, _, g, r, img = tr._forward(sc, learned=False)
    d_rgb, d_nrm = tr._loss(sc, img)
    l0 = float(tr.loss_dev.item())
    d = p2e_render_backward(g, r.proj, r.bins, sc.cams, r.cfg, img.alpha, img.last, d_rgb=d_rgb, d_normal=d_nrm)
    gr = d["rgb"]
    g.rgb[:, :3] -= 0.05 * gr / gr.abs().max()
    img = r.render(g, sc.cams)
    tr._loss(sc, img)
    l1 = float(tr.loss_dev.item())
    print(f"loss {l0:.5f} -> {l1:.5f} after a step on the colours")
    assert l1 < l0

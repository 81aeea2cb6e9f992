"""The usage example of the README runs as written (at 100K points and
512 x 512): a learned estimate of a cloud rendered for one camera, with
finite images and a covered figure."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_readme_usage_example():
    import scenes
    from paper_2409_16504_gb300 import Renderer, mlp
    from paper_2409_16504_gb300.estimate import LEARNED, Estimator, cloud_tensors

    xyz, rgb, _, _ = scenes.humanoid_cloud(100_000, seed=2)
    cx, cc = cloud_tensors(xyz, rgb)
    est = Estimator(len(xyz))
    gs = est(cx, cc, mode=LEARNED, mlp_blob=mlp.load_trained())
    cam = scenes.sphere_camera(xyz.mean(0), 2.5, np.random.default_rng(0), 512, 512)
    img = Renderer(capacity=1 << 22).render(gs, [cam])
    torch.cuda.synchronize()
    for k in ("rgb", "normal", "depth", "alpha"):
        assert bool(torch.isfinite(getattr(img, k)).all()), k
    cover = float((img.alpha > 0.5).float().mean())
    assert 0.02 < cover < 0.9, cover  # the figure fills part of the view

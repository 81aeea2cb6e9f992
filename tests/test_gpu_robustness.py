"""Robustness to voxelisation and density (the paper's quantised and
downsampled inputs, Sec. 3.3 and 4.2): on held-out scenes, the learned
estimator against kNN-PCA when the input cloud is 10-bit voxelised
(coarsened by alpha) or randomly subsampled (beta), the ground truth staying
exact.  The learned estimate stays ahead of kNN-PCA under every condition."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CONDITIONS = [None, ("quant", 1.0), ("quant", 0.5), ("quant", 0.25), ("sub", 0.25), ("sub", 0.125)]


def test_learned_stays_ahead_under_quantisation_and_subsampling():
    from paper_2409_16504_gb300 import mlp
    from paper_2409_16504_gb300.train import Scene, Trainer
    params = mlp.load_params()
    assert params is not None
    base = [Scene(2400 + s, 150_000, 6, 256) for s in range(2)]
    tr = Trainer(150_000, params=params)
    rows = {}
    for cond in CONDITIONS:
        scs = base if cond is None else [b.degraded(cond, seed=7 + k) for k, b in enumerate(base)]
        pca = float(np.mean([tr.evaluate(sc, learned=False)["psnr"] for sc in scs]))
        net = float(np.mean([tr.evaluate(sc, learned=True)["psnr"] for sc in scs]))
        pts = int(np.mean([sc.n for sc in scs]))
        rows["clean" if cond is None else f"{cond[0]} {cond[1]}"] = (pts, pca, net)
    print("\ncondition            points   kNN-PCA dB   learned dB")
    for k, (pts, pca, net) in rows.items():
        print(f"{k:18s} {pts:8d} {pca:11.2f} {net:12.2f}")
    for k, (_, pca, net) in rows.items():
        assert net > pca, (k, pca, net)

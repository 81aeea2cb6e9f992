"""Rendering quality against exact ground truth (Sec. 4.2 protocol on
synthetic stand-ins): the learned estimate must render within 0.1 dB of
the closed-form kNN-PCA estimate or better, on held-out scenes (12 views
on a circle at 512^2) and on the benchmark's 800K-point frame at 1024^2;
the comparison methods (global isotropic sizes, the point raster) are
reported beside them.  The full held-out set (16 scenes) is
``python -m paper_2409_16504_gb300.evaluate``."""
import pytest

pytestmark = pytest.mark.gpu


def _show(name, r):
    print(name, {k: (round(v, 2) if isinstance(v, float) else v) for k, v in r.items()})


def test_learned_within_0p1_db_of_knn_pca_held_out_512():
    from paper_2409_16504_gb300 import evaluate
    r = evaluate.held_out(range(2000, 2004), points=150_000, views=12, res=512)
    _show("held-out 4 x 12 views, 512^2:", r)
    assert r["learned"] >= r["knn_pca"] - 0.1
    assert r["knn_pca"] > r["global_1.7"] - 3.0  # sanity of the baselines


def test_learned_within_0p1_db_of_knn_pca_bench_frame_1024():
    from paper_2409_16504_gb300 import evaluate
    r = evaluate.bench_frame(points=800_000, res=1024, views=4)
    _show("bench frame 800K, 4 views, 1024^2:", r)
    assert r["learned"] >= r["knn_pca"] - 0.1

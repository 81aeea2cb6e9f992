"""The product's weight-blob packing equals the layout the oracle reads
(CPU: torch's bf16 rounding vs the oracle's explicit round-to-nearest-even)."""
import numpy as np
import torch

import oracle.mlp as om
from paper_2409_16504_gb300 import mlp


def test_pack_matches_oracle_layout():
    p = mlp.init_params(3, device="cpu")
    p["W4"] = torch.randn(mlp.OUT_PAD, mlp.HID) * 0.1
    p["W4"][mlp.OUT:] = 0
    for k in mlp.BIASES:
        p[k] = torch.randn(mlp.SHAPES[k])
    p["b4"][mlp.OUT:] = 0
    blob = mlp.pack(p).numpy()
    ref = om.pack_blob({k: v.double().numpy() for k, v in p.items()})
    np.testing.assert_array_equal(blob, ref)
    assert len(blob) == om.BLOB_BYTES == mlp.BLOB_BYTES

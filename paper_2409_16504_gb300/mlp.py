"""Weights of the learned per-point estimator (p2e_estimate mode 1).

The network (96 -> 64 -> 64 -> 64 -> 8, see include/p2e.h) runs in
libp2e's tcgen05 kernel; this module only lays out the weight blob the
kernel reads and loads trained weights shipped with the package."""
from __future__ import annotations

import os

import numpy as np
import torch

IN, HID, OUT, OUT_PAD = 96, 64, 8, 16
BLOB_BYTES = 31552
SHAPES = {"W1": (HID, IN), "W2": (HID, HID), "W3": (HID, HID), "W4": (OUT_PAD, HID),
          "b1": (HID,), "b2": (HID,), "b3": (HID,), "b4": (OUT_PAD,)}
WEIGHTS = ("W1", "W2", "W3", "W4")
BIASES = ("b1", "b2", "b3", "b4")
TRAINED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "estimator.npz")


def init_params(seed: int = 0, device="cuda") -> dict:
    """fp32 master parameters: He-initialised hidden layers, zero last layer
    (so the untrained network reproduces the PCA estimate)."""
    g = torch.Generator().manual_seed(seed)
    p = {}
    for k in WEIGHTS:
        o, i = SHAPES[k]
        p[k] = torch.randn((o, i), generator=g) * (2.0 / i) ** 0.5
    p["W4"].zero_()
    for k in BIASES:
        p[k] = torch.zeros(SHAPES[k])
    return {k: v.to(device) for k, v in p.items()}


def pack(params: dict) -> torch.Tensor:
    """Device byte blob: bf16 (round to nearest even) weights, fp32 biases."""
    dev = params["W1"].device
    parts = []
    for k in WEIGHTS:
        w = params[k].detach().to(torch.float32)
        if k == "W4":
            w = torch.cat([w[:OUT], torch.zeros((OUT_PAD - OUT, HID), device=dev)])
        parts.append(w.to(torch.bfloat16).contiguous().view(torch.uint8).reshape(-1))
    for k in BIASES:
        b = params[k].detach().to(torch.float32)
        if k == "b4":
            b = torch.cat([b[:OUT], torch.zeros(OUT_PAD - OUT, device=dev)])
        parts.append(b.contiguous().view(torch.uint8).reshape(-1))
    blob = torch.cat(parts)
    assert blob.numel() == BLOB_BYTES
    return blob


def save(params: dict, path: str = TRAINED):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.savez(path, **{k: v.detach().cpu().numpy() for k, v in params.items()})


def load_params(path: str = TRAINED, device="cuda") -> dict | None:
    if not os.path.exists(path):
        return None
    z = np.load(path)
    return {k: torch.from_numpy(z[k]).to(device) for k in SHAPES}


def load_trained(device="cuda") -> torch.Tensor | None:
    """Blob of the shipped trained weights, or None when none ship."""
    p = load_params(TRAINED, device)
    return None if p is None else pack(p)

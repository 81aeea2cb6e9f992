"""Python binding of p2e_estimate: argument marshalling only.

Point cloud (float4 xyz, float4 rgb on the device) in, one Gaussian per
point out (the preprocess stage of the paper's pipeline): mode 0 is the
closed-form kNN-PCA estimate, mode 1 adds the learned per-point MLP."""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from ._lib import check
from .render import GaussianSet, _ptr, _stream

PCA, LEARNED = 0, 1


class Estimator:
    """Owns the estimation scratch for clouds of up to ``n_max`` points."""

    def __init__(self, n_max: int, device="cuda"):
        self.device = device
        self.n_max = 0
        self._grow(n_max)

    def _grow(self, n: int):
        if n <= self.n_max:
            return
        sb = int(_lib.load().p2e_scratch_bytes(_lib.P2E_SCRATCH_ESTIMATE, n, 0))
        self.scratch = torch.empty((sb + 256,), dtype=torch.uint8, device=self.device)
        self.scratch_bytes = sb
        self.n_max = n

    def __call__(self, xyz: torch.Tensor, rgb: torch.Tensor, mode: int = PCA, opacity: float = 0.9,
                 mlp_blob: torch.Tensor | None = None, out: GaussianSet | None = None,
                 knn: torch.Tensor | None = None, stream=None) -> GaussianSet:
        n = xyz.shape[0]
        assert xyz.shape == (n, 4) and rgb.shape == (n, 4)
        self._grow(n)
        out = out or GaussianSet.empty(n, xyz.device)
        gs = out.c_struct()
        sp = (self.scratch.data_ptr() + 255) & ~255
        check("p2e_estimate", _lib.load().p2e_estimate(
            _ptr(xyz), _ptr(rgb), n, mode, _ptr(mlp_blob), C.c_float(opacity), C.byref(gs),
            _ptr(knn), C.c_void_p(sp), self.scratch_bytes, _stream(stream)))
        return out


    def check(self, n: int, stream=None) -> None:
        """Synchronises ``stream`` and raises if a bounded device wait of the
        last estimate on this scratch (``n`` points) gave up."""
        sp = (self.scratch.data_ptr() + 255) & ~255
        check("p2e_estimate", _lib.load().p2e_estimate_check(C.c_void_p(sp), self.scratch_bytes, n,
                                                             _stream(stream)))

    def global_(self, xyz: torch.Tensor, rgb: torch.Tensor, sigma_rel: float, opacity: float = 0.9,
                out: GaussianSet | None = None, knn: torch.Tensor | None = None, stream=None) -> GaussianSet:
        """The global isotropic baseline: scale sigma_rel x the cloud's mean
        nearest-neighbour distance for every point (p2e_estimate_global)."""
        n = xyz.shape[0]
        assert xyz.shape == (n, 4) and rgb.shape == (n, 4)
        self._grow(n)
        out = out or GaussianSet.empty(n, xyz.device)
        gs = out.c_struct()
        sp = (self.scratch.data_ptr() + 255) & ~255
        check("p2e_estimate_global", _lib.load().p2e_estimate_global(
            _ptr(xyz), _ptr(rgb), n, C.c_float(sigma_rel), C.c_float(opacity), C.byref(gs), _ptr(knn),
            C.c_void_p(sp), self.scratch_bytes, _stream(stream)))
        return out


def cloud_tensors(xyz, rgb, device="cuda"):
    """(n,3) numpy point/colour arrays -> float4 device tensors."""
    import numpy as np
    n = len(xyz)
    a = np.zeros((n, 4), np.float32)
    b = np.zeros((n, 4), np.float32)
    a[:, :3] = xyz
    b[:, :3] = rgb
    return torch.from_numpy(a).to(device), torch.from_numpy(b).to(device)

"""Python binding of the splatting renderer: argument marshalling only.

Every step of the path (projection, key emission, radix sort, tile ranges,
compositing, backward) runs in libp2e's CUDA kernels; PyTorch supplies
device memory and streams.  The low-level functions carry the C-ABI names
(``p2e_project``, ``p2e_sort_bin``, ``p2e_render``); :class:`Renderer` owns
reusable buffers and is what applications call.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import P2EBins, P2ECamera, P2EConfig, P2EGaussians, P2EProjected, check

DEFAULT_CONFIG = dict(tile=16, alpha_floor=1.0 / 255.0, alpha_max=0.99, t_min=1e-4, lowpass=0.3,
                      sigma_mult=3.0, bg=(0.0, 0.0, 0.0), schedule=0)


def _ptr(t: torch.Tensor | None):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def make_config(cfg: dict | None = None) -> P2EConfig:
    c = {**DEFAULT_CONFIG, **(cfg or {})}
    out = P2EConfig()
    out.tile = int(c["tile"])
    out.alpha_floor = c["alpha_floor"]
    out.alpha_max = c["alpha_max"]
    out.t_min = c["t_min"]
    out.lowpass = c["lowpass"]
    out.sigma_mult = c["sigma_mult"]
    for i in range(3):
        out.bg[i] = float(c["bg"][i])
    out.schedule = int(c.get("schedule", 0))
    return out


def make_cameras(cams: list) -> C.Array:
    arr = (P2ECamera * len(cams))()
    for k, cam in enumerate(cams):
        v = np.asarray(cam["viewmat"], np.float32).reshape(12)
        for i in range(12):
            arr[k].viewmat[i] = float(v[i])
        arr[k].fx, arr[k].fy = float(cam["fx"]), float(cam["fy"])
        arr[k].cx, arr[k].cy = float(cam["cx"]), float(cam["cy"])
        arr[k].width, arr[k].height = int(cam["width"]), int(cam["height"])
        arr[k].near_z = float(cam.get("near", 0.01))
    return arr


@dataclass
class GaussianSet:
    """Device Gaussian set in the float4 SoA layout of ``p2e_gaussians``."""
    mean_op: torch.Tensor   # (n, 4): x, y, z, opacity
    scale: torch.Tensor     # (n, 4)
    quat: torch.Tensor      # (n, 4): w, x, y, z
    rgb: torch.Tensor       # (n, 4)
    normal: torch.Tensor    # (n, 4)

    @property
    def n(self) -> int:
        return self.mean_op.shape[0]

    @staticmethod
    def empty(n: int, device="cuda") -> "GaussianSet":
        z = lambda: torch.zeros((n, 4), dtype=torch.float32, device=device)  # noqa: E731
        return GaussianSet(z(), z(), z(), z(), z())

    @staticmethod
    def from_numpy(g: dict, device="cuda") -> "GaussianSet":
        n = len(g["mean"])

        def pack(a, w=None):
            out = np.zeros((n, 4), np.float32)
            a = np.asarray(a, np.float32)
            out[:, : a.shape[1]] = a
            if w is not None:
                out[:, 3] = w
            return torch.from_numpy(out).to(device)

        return GaussianSet(pack(g["mean"], g["opacity"]), pack(g["scale"]), pack(g["quat"]),
                           pack(g["rgb"]), pack(g["normal"]))

    def c_struct(self) -> P2EGaussians:
        s = P2EGaussians()
        s.mean_op, s.scale, s.quat = self.mean_op.data_ptr(), self.scale.data_ptr(), self.quat.data_ptr()
        s.rgb, s.normal = self.rgb.data_ptr(), self.normal.data_ptr()
        s.n = self.n
        return s


class Projected:
    """Device buffers of ``p2e_projected`` for ``n_total`` (view, Gaussian) pairs."""

    def __init__(self, n_total: int, device="cuda"):
        self.xy_depth = torch.empty((max(n_total, 1), 4), dtype=torch.float32, device=device)
        self.conic_op = torch.empty((max(n_total, 1), 4), dtype=torch.float32, device=device)
        self.rect = torch.empty((max(n_total, 1), 4), dtype=torch.int16, device=device)
        self.ntiles = torch.empty((max(n_total, 1),), dtype=torch.int32, device=device)
        self.n_total = n_total

    def c_struct(self) -> P2EProjected:
        s = P2EProjected()
        s.xy_depth, s.conic_op = self.xy_depth.data_ptr(), self.conic_op.data_ptr()
        s.rect, s.ntiles = self.rect.data_ptr(), self.ntiles.data_ptr()
        return s


class Bins:
    """Device buffers of ``p2e_bins``."""

    def __init__(self, n_total: int, total_tiles: int, capacity: int, device="cuda"):
        lib = _lib.load()
        cap = max(int(capacity), 1)
        self.keys = [torch.empty((cap,), dtype=torch.int64, device=device) for _ in range(2)]
        self.vals = [torch.empty((cap,), dtype=torch.int32, device=device) for _ in range(2)]
        self.ranges = torch.zeros((max(total_tiles, 1), 2), dtype=torch.int32, device=device)
        self.tile_work = torch.zeros((total_tiles + 2,), dtype=torch.int32, device=device)
        sb = int(lib.p2e_scratch_bytes(_lib.P2E_SCRATCH_SORT, n_total, cap))
        self.scratch = torch.empty((sb + 256,), dtype=torch.uint8, device=device)
        self.counters = torch.zeros((2,), dtype=torch.int64, device=device)  # n_keys, status
        self.capacity, self.n_total, self.total_tiles = cap, n_total, total_tiles
        self.struct = P2EBins()
        s = self.struct
        s.keys[0], s.keys[1] = self.keys[0].data_ptr(), self.keys[1].data_ptr()
        s.vals[0], s.vals[1] = self.vals[0].data_ptr(), self.vals[1].data_ptr()
        s.ranges = self.ranges.data_ptr()
        s.tile_work = self.tile_work.data_ptr()
        base = self.scratch.data_ptr()
        s.scratch = (base + 255) & ~255
        s.scratch_bytes = sb
        s.capacity = cap
        s.n_keys_dev = self.counters.data_ptr()
        s.status_dev = self.counters.data_ptr() + 8
        s.result = 0

    def fits(self, n_total, total_tiles, capacity):
        return n_total <= self.n_total and total_tiles <= self.total_tiles and capacity <= self.capacity

    def sorted(self):
        r = self.struct.result
        return self.keys[r], self.vals[r]


# ---------------------------------------------------------------- C-ABI calls
def p2e_project(g: GaussianSet, cams: list, cfg: dict | None, out: Projected, stream=None):
    lib = _lib.load()
    ca = make_cameras(cams)
    gs, ps, cf = g.c_struct(), out.c_struct(), make_config(cfg)
    check("p2e_project", lib.p2e_project(C.byref(gs), ca, len(cams), C.byref(cf), C.byref(ps),
                                         _stream(stream)))


def p2e_sort_bin(proj: Projected, n: int, cams: list, cfg: dict | None, bins: Bins, stream=None):
    lib = _lib.load()
    ca = make_cameras(cams)
    ps, cf = proj.c_struct(), make_config(cfg)
    check("p2e_sort_bin", lib.p2e_sort_bin(C.byref(ps), n, ca, len(cams), C.byref(cf),
                                           C.byref(bins.struct), _stream(stream)))


def p2e_bins_check(bins: Bins, stream=None) -> tuple[int, int]:
    """Synchronises; returns (status, key count)."""
    lib = _lib.load()
    k = C.c_int64(0)
    st = lib.p2e_bins_check(C.byref(bins.struct), C.byref(k), _stream(stream))
    return int(st), int(k.value)


def p2e_render(g: GaussianSet, proj: Projected, bins: Bins, cams: list, cfg: dict | None,
               rgb=None, normal=None, depth=None, alpha=None, last=None, stream=None):
    lib = _lib.load()
    ca = make_cameras(cams)
    gs, ps, cf = g.c_struct(), proj.c_struct(), make_config(cfg)
    check("p2e_render", lib.p2e_render(C.byref(gs), C.byref(ps), C.byref(bins.struct), ca, len(cams),
                                       C.byref(cf), _ptr(rgb), _ptr(normal), _ptr(depth), _ptr(alpha),
                                       _ptr(last), _stream(stream)))


def total_tiles(cams: list, tile: int) -> int:
    ca = make_cameras(cams)
    t = int(_lib.load().p2e_total_tiles(ca, len(cams), tile))
    if t < 0:
        raise _lib.P2EError("p2e_total_tiles", _lib.P2E_ERR_INVALID_ARG)
    return t


# ---------------------------------------------------------------- high level
class Images:
    """Planar outputs of one render call (views concatenated)."""

    def __init__(self, cams: list, device="cuda"):
        self.sizes = [(int(c["height"]), int(c["width"])) for c in cams]
        npix = sum(h * w for h, w in self.sizes)
        self.npix = npix
        self.rgb = torch.empty((3 * npix,), dtype=torch.float32, device=device)
        self.normal = torch.empty((3 * npix,), dtype=torch.float32, device=device)
        self.depth = torch.empty((npix,), dtype=torch.float32, device=device)
        self.alpha = torch.empty((npix,), dtype=torch.float32, device=device)
        self.last = torch.empty((npix,), dtype=torch.int32, device=device)

    def view(self, v: int) -> dict:
        off = sum(h * w for h, w in self.sizes[:v])
        h, w = self.sizes[v]
        return dict(rgb=self.rgb[3 * off: 3 * off + 3 * h * w].view(3, h, w),
                    normal=self.normal[3 * off: 3 * off + 3 * h * w].view(3, h, w),
                    depth=self.depth[off: off + h * w].view(h, w),
                    alpha=self.alpha[off: off + h * w].view(h, w),
                    last=self.last[off: off + h * w].view(h, w))


class Renderer:
    """Owns projection, binning and image buffers; renders batches of views.

    ``capacity`` is the key capacity; when a frame needs more keys the buffers
    grow (by 1.5x the need) and the frame is re-rendered (``render`` with
    ``check=True``).  ``render(check=False)`` never synchronises.
    """

    def __init__(self, cfg: dict | None = None, capacity: int = 1 << 20, device="cuda"):
        self.cfg = {**DEFAULT_CONFIG, **(cfg or {})}
        self.device = device
        self.capacity = int(capacity)
        self.proj: Projected | None = None
        self.bins: Bins | None = None
        self.n_keys = 0

    def _ensure(self, n_total, tt):
        if self.proj is None or self.proj.n_total < n_total:
            self.proj = Projected(n_total, self.device)
        if self.bins is None or not self.bins.fits(n_total, tt, self.capacity):
            self.bins = Bins(n_total, tt, self.capacity, self.device)

    def render(self, g: GaussianSet, cams: list, out: Images | None = None, check: bool = True,
               stream=None) -> Images:
        tt = total_tiles(cams, self.cfg["tile"])
        self._ensure(g.n * len(cams), tt)
        out = out or Images(cams, self.device)
        for _ in range(3):
            p2e_project(g, cams, self.cfg, self.proj, stream)
            p2e_sort_bin(self.proj, g.n, cams, self.cfg, self.bins, stream)
            p2e_render(g, self.proj, self.bins, cams, self.cfg, out.rgb, out.normal, out.depth,
                       out.alpha, out.last, stream)
            if not check:
                return out
            st, k = p2e_bins_check(self.bins, stream)
            self.n_keys = k
            if st == _lib.P2E_OK:
                return out
            if st != _lib.P2E_ERR_CAPACITY:
                raise _lib.P2EError("p2e_sort_bin / p2e_render", st)
            self.capacity = int(k * 1.5) + 1024
            self._ensure(g.n * len(cams), tt)
        raise _lib.P2EError("p2e_sort_bin", _lib.P2E_ERR_CAPACITY)


def relight(img: Images, lights, ambient: float = 0.2, bg=(0.0, 0.0, 0.0), out: torch.Tensor | None = None,
            stream=None) -> torch.Tensor:
    """Late shading of rendered views from their normal images
    (p2e_relight): Lambertian directional lights plus ambient.  ``lights``:
    sequence of (dx, dy, dz, intensity) in the normals' world frame.  Returns
    the planar rgb of all views (``out`` may be ``img.rgb``)."""
    lib = _lib.load()
    lt = [float(v) for l4 in lights for v in l4]
    if len(lt) % 4:
        raise ValueError("lights are (dx, dy, dz, intensity) tuples")
    la = (C.c_float * max(len(lt), 1))(*lt)
    bga = (C.c_float * 3)(*[float(b) for b in bg])
    vp = (C.c_int64 * len(img.sizes))(*[h * w for h, w in img.sizes])
    out = out if out is not None else torch.empty_like(img.rgb)
    check("p2e_relight", lib.p2e_relight(_ptr(img.rgb), _ptr(img.normal), _ptr(img.alpha), vp, len(img.sizes), la,
                                         len(lt) // 4, C.c_float(ambient), bga, _ptr(out), _stream(stream)))
    return out


def point_raster(xyz: torch.Tensor, rgb: torch.Tensor, cams: list, bg=(0.0, 0.0, 0.0), out: Images | None = None,
                 stream=None) -> Images:
    """The 1-pixel point-rasterisation baseline (p2e_point_raster) of a
    float4 cloud: rgb and depth planes of every view (alpha, normal and
    last of ``out`` are left untouched)."""
    lib = _lib.load()
    n = xyz.shape[0]
    out = out or Images(cams, xyz.device)
    zbuf = torch.empty((out.npix,), dtype=torch.int64, device=xyz.device)
    ca = make_cameras(cams)
    bga = (C.c_float * 3)(*[float(b) for b in bg])
    check("p2e_point_raster", lib.p2e_point_raster(_ptr(xyz), _ptr(rgb), n, ca, len(cams), bga, _ptr(zbuf),
                                                   _ptr(out.rgb), _ptr(out.depth), _stream(stream)))
    return out


# ---------------------------------------------------------------- backward
def p2e_render_backward(g: GaussianSet, proj: Projected, bins: Bins, cams: list, cfg: dict | None,
                        alpha: torch.Tensor, last: torch.Tensor, d_rgb=None, d_normal=None,
                        d_depth=None, d_alpha=None, stream=None) -> dict:
    """Gradients (w.r.t. mean, scale, raw quaternion, opacity, rgb, normal)
    of <upstream, images> for the render that produced ``alpha``/``last``."""
    lib = _lib.load()
    ca = make_cameras(cams)
    gs, ps, cf = g.c_struct(), proj.c_struct(), make_config(cfg)
    n = g.n
    dev = g.mean_op.device
    out = dict(mean=torch.empty((n, 3), dtype=torch.float32, device=dev),
               scale=torch.empty((n, 3), dtype=torch.float32, device=dev),
               quat=torch.empty((n, 4), dtype=torch.float32, device=dev),
               opacity=torch.empty((n,), dtype=torch.float32, device=dev),
               rgb=torch.empty((n, 3), dtype=torch.float32, device=dev),
               normal=torch.empty((n, 3), dtype=torch.float32, device=dev))
    sb = int(lib.p2e_scratch_bytes(_lib.P2E_SCRATCH_BACKWARD, n * len(cams), 0))
    scratch = torch.empty((sb + 256,), dtype=torch.uint8, device=dev)
    sp = (scratch.data_ptr() + 255) & ~255
    check("p2e_render_backward", lib.p2e_render_backward(
        C.byref(gs), C.byref(ps), C.byref(bins.struct), ca, len(cams), C.byref(cf), _ptr(alpha),
        _ptr(last), _ptr(d_rgb), _ptr(d_normal), _ptr(d_depth), _ptr(d_alpha), _ptr(out["mean"]),
        _ptr(out["scale"]), _ptr(out["quat"]), _ptr(out["opacity"]), _ptr(out["rgb"]),
        _ptr(out["normal"]), C.c_void_p(sp), sb, _stream(stream)))
    return out


class _RenderFn(torch.autograd.Function):
    """Differentiable render of float4-SoA Gaussian tensors (see
    :func:`render_differentiable`)."""

    @staticmethod
    def forward(ctx, mean_op, scale, quat, rgb, normal, cams, cfg):
        gs = GaussianSet(mean_op.detach().contiguous(), scale.detach().contiguous(),
                         quat.detach().contiguous(), rgb.detach().contiguous(),
                         normal.detach().contiguous())
        r = Renderer(cfg, capacity=max(1 << 16, 4 * gs.n * len(cams)), device=mean_op.device)
        img = r.render(gs, cams)
        ctx.state = (gs, r, img, cams, cfg)
        return img.rgb, img.normal, img.depth, img.alpha

    @staticmethod
    def backward(ctx, g_rgb, g_normal, g_depth, g_alpha):
        gs, r, img, cams, cfg = ctx.state
        c = lambda t: None if t is None else t.contiguous()  # noqa: E731
        d = p2e_render_backward(gs, r.proj, r.bins, cams, r.cfg, img.alpha, img.last, c(g_rgb),
                                c(g_normal), c(g_depth), c(g_alpha))
        z = torch.zeros((gs.n, 1), dtype=torch.float32, device=gs.mean_op.device)
        ctx.state = None
        return (torch.cat([d["mean"], d["opacity"][:, None]], 1), torch.cat([d["scale"], z], 1),
                d["quat"], torch.cat([d["rgb"], z], 1), torch.cat([d["normal"], z], 1), None, None)


def render_differentiable(mean_op, scale, quat, rgb, normal, cams: list, cfg: dict | None = None):
    """Render views from float4-SoA Gaussian tensors with autograd support.

    Returns planar (rgb, normal, depth, alpha) tensors, views concatenated
    (see :class:`Images`).  Gradients flow to all five inputs (the opacity
    is column 3 of ``mean_op``; the unused fourth columns get zeros).
    """
    return _RenderFn.apply(mean_op, scale, quat, rgb, normal, cams, {**DEFAULT_CONFIG, **(cfg or {})})

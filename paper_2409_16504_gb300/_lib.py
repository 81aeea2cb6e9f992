"""ctypes loader of libp2e.so and the C structs of include/p2e.h.

The library is built in-tree (``paper_2409_16504_gb300/_build/libp2e.so``)
by :func:`paper_2409_16504_gb300.build.build`.  There is no fallback: if the
library cannot be loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

P2E_OK, P2E_ERR_INVALID_ARG, P2E_ERR_CAPACITY, P2E_ERR_CUDA, P2E_ERR_TIMEOUT, P2E_ERR_UNSUPPORTED = range(6)
P2E_MAX_VIEWS = 64
P2E_SCHEDULE_AUTO, P2E_SCHEDULE_PER_BLOCK = 0, 1
P2E_SCRATCH_SORT, P2E_SCRATCH_ESTIMATE, P2E_SCRATCH_BACKWARD = 0, 1, 2

# every symbol include/p2e.h declares
EXPORTS = ("p2e_default_config", "p2e_total_tiles", "p2e_scratch_bytes", "p2e_project",
           "p2e_sort_bin", "p2e_sort_bin_noalloc", "p2e_bins_check", "p2e_render",
           "p2e_render_backward", "p2e_estimate", "p2e_loss_eq5", "p2e_mlp_backward", "p2e_adam",
           "p2e_estimate_global", "p2e_relight", "p2e_point_raster", "p2e_set_kernel_probe",
           "p2e_estimate_check", "p2e_selftest_timeout", "p2e_loss_ssim", "p2e_loss_splat_area",
           "p2e_status_string")
P2E_PROBE_KNN, P2E_PROBE_BLEND, P2E_PROBE_MLP, P2E_PROBE_BLEND_BWD = 0, 1, 2, 3
SELFTEST_SCRATCH_BYTES = 1 << 20
P2E_MAX_LIGHTS = 8
MLP_PARAMS = 15568
NOALLOC_MAX_N = 1 << 22
NOALLOC_MAX_CAPACITY = 1 << 21


class P2ECamera(C.Structure):
    _fields_ = [("viewmat", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_z", C.c_float)]


class P2EConfig(C.Structure):
    _fields_ = [("tile", C.c_int32), ("alpha_floor", C.c_float), ("alpha_max", C.c_float),
                ("t_min", C.c_float), ("lowpass", C.c_float), ("sigma_mult", C.c_float),
                ("bg", C.c_float * 3), ("schedule", C.c_int32)]


class P2EGaussians(C.Structure):
    _fields_ = [("mean_op", C.c_void_p), ("scale", C.c_void_p), ("quat", C.c_void_p),
                ("rgb", C.c_void_p), ("normal", C.c_void_p), ("n", C.c_int64)]


class P2EProjected(C.Structure):
    _fields_ = [("xy_depth", C.c_void_p), ("conic_op", C.c_void_p), ("rect", C.c_void_p),
                ("ntiles", C.c_void_p)]


class P2EBins(C.Structure):
    _fields_ = [("keys", C.c_void_p * 2), ("vals", C.c_void_p * 2), ("ranges", C.c_void_p),
                ("tile_work", C.c_void_p), ("scratch", C.c_void_p), ("scratch_bytes", C.c_int64), ("capacity", C.c_int64),
                ("n_keys_dev", C.c_void_p), ("status_dev", C.c_void_p), ("result", C.c_int32)]


class P2EKernelProbe(C.Structure):
    _fields_ = [("start_event", C.c_void_p), ("stop_event", C.c_void_p), ("count_dev", C.c_void_p)]


class P2EError(RuntimeError):
    def __init__(self, fn: str, status: int):
        self.status = status
        super().__init__(f"{fn}: {status_string(status)} (status {status})")


def load(path: str | None = None):
    """Load (building first if needed) libp2e.so."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib_path = path or _build.LIB
        if not os.path.exists(lib_path):
            _build.build()
        lib = C.CDLL(lib_path)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        lib.p2e_default_config.restype = P2EConfig
        lib.p2e_default_config.argtypes = []
        lib.p2e_total_tiles.restype = i64
        lib.p2e_total_tiles.argtypes = [C.POINTER(P2ECamera), i32, i32]
        lib.p2e_scratch_bytes.restype = C.c_size_t
        lib.p2e_scratch_bytes.argtypes = [i32, i64, i64]
        lib.p2e_status_string.restype = C.c_char_p
        lib.p2e_status_string.argtypes = [C.c_int]
        lib.p2e_project.restype = C.c_int
        lib.p2e_project.argtypes = [C.POINTER(P2EGaussians), C.POINTER(P2ECamera), i32,
                                    C.POINTER(P2EConfig), C.POINTER(P2EProjected), vp]
        lib.p2e_sort_bin.restype = C.c_int
        lib.p2e_sort_bin.argtypes = [C.POINTER(P2EProjected), i64, C.POINTER(P2ECamera), i32,
                                     C.POINTER(P2EConfig), C.POINTER(P2EBins), vp]
        lib.p2e_sort_bin_noalloc.restype = C.c_int
        lib.p2e_sort_bin_noalloc.argtypes = [C.POINTER(P2EProjected), i64, C.POINTER(P2ECamera), i32,
                                             C.POINTER(P2EConfig), C.POINTER(P2EBins), vp]
        lib.p2e_bins_check.restype = C.c_int
        lib.p2e_bins_check.argtypes = [C.POINTER(P2EBins), C.POINTER(C.c_int64), vp]
        lib.p2e_render.restype = C.c_int
        lib.p2e_render.argtypes = [C.POINTER(P2EGaussians), C.POINTER(P2EProjected),
                                   C.POINTER(P2EBins), C.POINTER(P2ECamera), i32,
                                   C.POINTER(P2EConfig), vp, vp, vp, vp, vp, vp]
        lib.p2e_render_backward.restype = C.c_int
        lib.p2e_render_backward.argtypes = [C.POINTER(P2EGaussians), C.POINTER(P2EProjected),
                                            C.POINTER(P2EBins), C.POINTER(P2ECamera), i32,
                                            C.POINTER(P2EConfig), vp, vp, vp, vp, vp, vp,
                                            vp, vp, vp, vp, vp, vp, vp, i64, vp]
        lib.p2e_estimate.restype = C.c_int
        lib.p2e_estimate.argtypes = [vp, vp, i64, i32, vp, C.c_float, C.POINTER(P2EGaussians),
                                     vp, vp, i64, vp]
        lib.p2e_loss_eq5.restype = C.c_int
        lib.p2e_loss_eq5.argtypes = [vp, vp, vp, vp, C.POINTER(C.c_int64), i32, C.c_float, C.c_float,
                                     C.c_float, vp, vp, vp, vp]
        lib.p2e_mlp_backward.restype = C.c_int
        lib.p2e_mlp_backward.argtypes = [vp, vp, i64, vp, C.POINTER(P2EGaussians), vp, vp, vp, vp, vp,
                                         vp, vp]
        lib.p2e_adam.restype = C.c_int
        lib.p2e_adam.argtypes = [vp, vp, vp, vp, i64, C.c_float, C.c_float, C.c_float, C.c_float, i32,
                                 vp, vp]
        lib.p2e_estimate_global.restype = C.c_int
        lib.p2e_estimate_global.argtypes = [vp, vp, i64, C.c_float, C.c_float, C.POINTER(P2EGaussians), vp, vp,
                                            i64, vp]
        lib.p2e_relight.restype = C.c_int
        lib.p2e_relight.argtypes = [vp, vp, vp, C.POINTER(C.c_int64), i32, C.POINTER(C.c_float), i32, C.c_float,
                                    C.POINTER(C.c_float), vp, vp]
        lib.p2e_point_raster.restype = C.c_int
        lib.p2e_point_raster.argtypes = [vp, vp, i64, C.POINTER(P2ECamera), i32, C.POINTER(C.c_float), vp, vp, vp,
                                         vp]
        lib.p2e_set_kernel_probe.restype = C.c_int
        lib.p2e_set_kernel_probe.argtypes = [i32, C.POINTER(P2EKernelProbe)]
        lib.p2e_estimate_check.restype = C.c_int
        lib.p2e_estimate_check.argtypes = [vp, i64, i64, vp]
        lib.p2e_loss_ssim.restype = C.c_int
        lib.p2e_loss_ssim.argtypes = [vp, vp, C.POINTER(C.c_int32), i32, C.c_float, vp, vp, vp, i64, vp]
        lib.p2e_loss_splat_area.restype = C.c_int
        lib.p2e_loss_splat_area.argtypes = [vp, vp, i64, C.c_float, vp, vp, vp]
        lib.p2e_selftest_timeout.restype = C.c_int
        lib.p2e_selftest_timeout.argtypes = [i32, C.c_uint32, vp, i64, vp, vp]
        _lib = lib
        return lib


def status_string(s: int) -> str:
    return load().p2e_status_string(int(s)).decode()


def check(fn: str, status: int):
    if status != P2E_OK:
        raise P2EError(fn, status)

"""The C ABI's argument validation, on a machine without a GPU.

Every entry point of include/p2e.h checks its arguments on the host and
returns P2E_ERR_INVALID_ARG before any CUDA call or launch.  Each case
below is invalid in exactly one way and otherwise well formed.  The device
addresses are fake: 16- or 256-byte aligned integers the library must never
dereference, because validation rejects the call first.  Host structs
(cameras, configurations, Gaussian and bin descriptors) are real.
"""
import ctypes as C
import math

import pytest

from paper_2409_16504_gb300 import _lib

OK, INVALID = _lib.P2E_OK, _lib.P2E_ERR_INVALID_ARG
A = 0x7f0000000000          # a fake, 256-byte aligned device address
MIS = A + 8                 # the same, off the 16-byte boundary


def lib():
    return _lib.load()


def cams(n=1, **over):
    arr = (_lib.P2ECamera * n)()
    for c in arr:
        vm = [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 3]
        for i in range(12):
            c.viewmat[i] = vm[i]
        c.fx = c.fy = 100.0
        c.cx, c.cy = 64.0, 64.0
        c.width = c.height = 128
        c.near_z = 0.01
        for k, v in over.items():
            if k == "viewmat0":
                c.viewmat[0] = v
            else:
                setattr(c, k, v)
    return arr


def cfg(**over):
    c = lib().p2e_default_config()
    for k, v in over.items():
        setattr(c, k, v)
    return c


def gauss(n=100, **over):
    g = _lib.P2EGaussians(A, A + 0x1000, A + 0x2000, A + 0x3000, A + 0x4000, n)
    for k, v in over.items():
        setattr(g, k, v)
    return g


def proj(**over):
    p = _lib.P2EProjected(A + 0x5000, A + 0x6000, A + 0x7000, A + 0x8000)
    for k, v in over.items():
        setattr(p, k, v)
    return p


def bins(**over):
    b = _lib.P2EBins()
    b.keys[0], b.keys[1] = A + 0x10000, A + 0x20000
    b.vals[0], b.vals[1] = A + 0x30000, A + 0x40000
    b.ranges, b.tile_work, b.scratch = A + 0x50000, A + 0x60000, A + 0x100000
    b.scratch_bytes, b.capacity = 1 << 30, 1 << 20
    b.n_keys_dev, b.status_dev, b.result = A + 0x70000, A + 0x80000, 0
    for k, v in over.items():
        setattr(b, k, v)
    return b


# ---------------------------------------------------------------- project
@pytest.mark.parametrize("case", [
    dict(g=None), dict(g=dict(n=-1)), dict(g=dict(n=1 << 31)), dict(g=dict(scale=None)),
    dict(g=dict(mean_op=MIS)), dict(g=dict(normal=A + 4)),
    dict(views=0), dict(views=_lib.P2E_MAX_VIEWS + 1),
    dict(cfg=dict(tile=12)), dict(cfg=dict(tile=64)), dict(cfg=dict(alpha_max=1.5)),
    dict(cfg=dict(alpha_max=0.0)), dict(cfg=dict(alpha_floor=-0.1)), dict(cfg=dict(t_min=1.0)),
    dict(cfg=dict(lowpass=-0.3)), dict(cfg=dict(lowpass=math.nan)), dict(cfg=dict(sigma_mult=0.0)),
    dict(cfg=dict(schedule=7)),
    dict(cam=dict(width=0)), dict(cam=dict(height=8193)), dict(cam=dict(fx=math.inf)),
    dict(cam=dict(near_z=-1.0)), dict(cam=dict(viewmat0=math.nan)),
    dict(out=None), dict(out=dict(xy_depth=MIS)), dict(out=dict(rect=A + 4)), dict(out=dict(ntiles=A + 2)),
])
def test_project_rejects(case):
    g = None if case.get("g", 0) is None else gauss(**case.get("g", {}))
    nv = case.get("views", 1)
    cm = cams(max(nv, 1), **case.get("cam", {}))
    o = None if case.get("out", 0) is None else proj(**case.get("out", {}))
    st = lib().p2e_project(C.byref(g) if g is not None else None, cm, nv, C.byref(cfg(**case.get("cfg", {}))),
                           C.byref(o) if o is not None else None, None)
    assert st == INVALID


def test_project_null_camera_and_config():
    g, o = gauss(), proj()
    assert lib().p2e_project(C.byref(g), None, 1, C.byref(cfg()), C.byref(o), None) == INVALID
    assert lib().p2e_project(C.byref(g), cams(), 1, None, C.byref(o), None) == INVALID


def test_total_tiles_at_the_largest_views():
    """64 views of 8192 x 8192 at 8-px tiles: 2^26 tile ids, counted in 64
    bits; an unsupported tile size or no views gives -1."""
    c = cams(_lib.P2E_MAX_VIEWS, width=8192, height=8192)
    assert lib().p2e_total_tiles(c, _lib.P2E_MAX_VIEWS, 8) == _lib.P2E_MAX_VIEWS * 1024 * 1024
    assert lib().p2e_total_tiles(c, _lib.P2E_MAX_VIEWS, 12) == -1
    assert lib().p2e_total_tiles(c, 0, 16) == -1


# ---------------------------------------------------------------- sort_bin
@pytest.mark.parametrize("case", [
    dict(n=-1), dict(n=1 << 31), dict(io=None), dict(views=0),
    dict(proj=None), dict(proj=dict(conic_op=MIS)),
    dict(io=dict(capacity=-1)), dict(io=dict(capacity=1 << 30)), dict(io=dict(ranges=None)),
    dict(io=dict(tile_work=None)), dict(io=dict(n_keys_dev=None)), dict(io=dict(status_dev=None)),
    dict(io=dict(scratch=None)), dict(io=dict(scratch=A + 128)), dict(io=dict(ranges=A + 4)),
    dict(io=dict(scratch_bytes=1024)), dict(io=dict(keys=(C.c_void_p * 2)(A, 0))),
])
def test_sort_bin_rejects(case):
    n = case.get("n", 1000)
    io = None if case.get("io", 0) is None else bins(**case.get("io", {}))
    p = None if case.get("proj", 0) is None else proj(**case.get("proj", {}))
    nv = case.get("views", 1)
    st = lib().p2e_sort_bin(C.byref(p) if p is not None else None, n, cams(max(nv, 1)), nv,
                            C.byref(cfg(tile=8)), C.byref(io) if io is not None else None, None)
    assert st == INVALID


@pytest.mark.parametrize("case", [dict(n=-1), dict(views=0), dict(views=_lib.P2E_MAX_VIEWS + 1),
                                  dict(io=None), dict(capacity=-1)])
def test_noalloc_rejects(case):
    """The allocation-free binning checks n, the views and the capacity on
    the host before it looks up its device array; the rest of its arguments
    go through p2e_sort_bin's checks."""
    io = None if "io" in case else bins(capacity=case.get("capacity", 1 << 20))
    nv = case.get("views", 1)
    st = lib().p2e_sort_bin_noalloc(C.byref(proj()), case.get("n", 1000), cams(max(nv, 1)), nv,
                                    C.byref(cfg()), C.byref(io) if io is not None else None, None)
    assert st == INVALID


def test_noalloc_limits():
    """The allocation-free binning refuses work beyond its fixed array."""
    f = lib().p2e_sort_bin_noalloc
    p, b = proj(), bins(capacity=1 << 20)
    assert f(C.byref(p), _lib.NOALLOC_MAX_N + 1, cams(), 1, C.byref(cfg()), C.byref(b), None) == INVALID
    # n within the limit, n x views beyond it (n is bounded before the product)
    assert f(C.byref(p), _lib.NOALLOC_MAX_N // 2 + 1, cams(2), 2, C.byref(cfg()), C.byref(b), None) == INVALID
    b.capacity = _lib.NOALLOC_MAX_CAPACITY + 1
    assert f(C.byref(p), 1000, cams(), 1, C.byref(cfg()), C.byref(b), None) == INVALID


def test_bins_check_rejects_missing_words():
    f = lib().p2e_bins_check
    assert f(None, None, None) == INVALID
    for k in ("n_keys_dev", "status_dev"):
        b = bins(**{k: None})
        assert f(C.byref(b), None, None) == INVALID


# ---------------------------------------------------------------- render
@pytest.mark.parametrize("case", [
    dict(g=dict(quat=None)), dict(bins=None), dict(bins=dict(result=2)), dict(bins=dict(ranges=None)),
    dict(bins=dict(tile_work=None)), dict(bins=dict(vals=(C.c_void_p * 2)(0, A))),
    dict(proj=dict(ntiles=None)), dict(cfg=dict(bg=(C.c_float * 3)(0, math.nan, 0))),
])
def test_render_rejects(case):
    g = gauss(**case.get("g", {}))
    p = proj(**case.get("proj", {}))
    b = None if case.get("bins", 0) is None else bins(**case.get("bins", {}))
    planes = [A + 0x200000 * k for k in range(1, 6)]
    st = lib().p2e_render(C.byref(g), C.byref(p), C.byref(b) if b is not None else None, cams(), 1,
                          C.byref(cfg(**case.get("cfg", {}))), *planes, None)
    assert st == INVALID


@pytest.mark.parametrize("case", [
    dict(last=None), dict(bins=dict(result=-1)), dict(grad=2), dict(scratch_bytes=16),
    dict(scratch=A + 64), dict(g=dict(rgb=MIS)),
])
def test_render_backward_rejects(case):
    g = gauss(**case.get("g", {}))
    p, b = proj(), bins(**case.get("bins", {}))
    ups = [A + 0x200000 * k for k in range(1, 5)]
    grads = [A + 0x1000000 + 0x100000 * k for k in range(6)]
    if "grad" in case:
        grads[case["grad"]] = None
    last = case.get("last", A + 0x3000000)
    scratch = case.get("scratch", A + 0x4000000)
    sb = case.get("scratch_bytes", 1 << 30)
    st = lib().p2e_render_backward(C.byref(g), C.byref(p), C.byref(b), cams(), 1, C.byref(cfg()),
                                   A + 0x2000000, last, *ups, *grads, scratch, sb, None)
    assert st == INVALID


# ---------------------------------------------------------------- estimate
def _est(fn="p2e_estimate", n=1000, mode=0, weights=A + 0x9000000, opacity=0.9, xyz=A, rgb=A + 0x1000000,
         out=0, knn=None, scratch=A + 0x2000000, sb=1 << 34, sigma=1.2):
    o = gauss() if out == 0 else out
    po = C.byref(o) if o is not None else None
    if fn == "p2e_estimate":
        return lib().p2e_estimate(xyz, rgb, n, mode, weights, opacity, po, knn, scratch, sb, None)
    return lib().p2e_estimate_global(xyz, rgb, n, sigma, opacity, po, knn, scratch, sb, None)


@pytest.mark.parametrize("fn", ["p2e_estimate", "p2e_estimate_global"])
@pytest.mark.parametrize("case", [
    dict(n=-1), dict(n=1 << 31), dict(n=16), dict(n=1), dict(out=None), dict(opacity=1.5),
    dict(opacity=-0.1), dict(opacity=math.nan), dict(xyz=None), dict(xyz=MIS), dict(rgb=A + 4),
    dict(out=gauss(scale=None)), dict(out=gauss(quat=MIS)), dict(scratch=None),
    dict(scratch=A + 128), dict(sb=1024), dict(knn=MIS),
])
def test_estimate_rejects(fn, case):
    assert _est(fn, **case) == INVALID


def test_estimate_mode_and_weights():
    assert _est(mode=2) == INVALID
    assert _est(mode=-1) == INVALID
    assert _est(mode=1, weights=None) == INVALID          # the learned head needs its weights
    assert _est("p2e_estimate_global", sigma=0.0) == INVALID
    assert _est("p2e_estimate_global", sigma=math.inf) == INVALID


def test_estimate_of_nothing_is_ok():
    """An empty cloud is a valid call that launches nothing."""
    assert _est(n=0, xyz=None, rgb=None, scratch=None, sb=0) == OK
    assert _est("p2e_estimate_global", n=0, xyz=None, rgb=None, scratch=None, sb=0) == OK


def test_estimate_check_rejects():
    f = lib().p2e_estimate_check
    assert f(A, 1 << 34, 16, None) == INVALID
    assert f(None, 1 << 34, 1000, None) == INVALID
    assert f(A + 128, 1 << 34, 1000, None) == INVALID
    assert f(A, 1024, 1000, None) == INVALID


def test_scratch_sizes_grow_with_the_work():
    f = lib().p2e_scratch_bytes
    for kind in (_lib.P2E_SCRATCH_SORT, _lib.P2E_SCRATCH_ESTIMATE, _lib.P2E_SCRATCH_BACKWARD):
        a, b = f(kind, 1000, 1 << 16), f(kind, 100_000, 1 << 20)
        assert 0 < a <= b
    assert f(7, 1000, 1000) == 0 and f(0, -1, 1000) == 0 and f(0, 1000, -1) == 0


# ---------------------------------------------------------------- training
def test_loss_eq5_rejects():
    f = lib().p2e_loss_eq5
    px = (C.c_int64 * 2)(100, 100)
    bufs = [A + 0x100000 * k for k in range(4)]
    outs = [A + 0x1000000 + 0x100000 * k for k in range(3)]
    assert f(*bufs, px, 0, 1.0, 0.1, 0.1, *outs, None) == INVALID
    assert f(*bufs, px, _lib.P2E_MAX_VIEWS + 1, 1.0, 0.1, 0.1, *outs, None) == INVALID
    assert f(None, *bufs[1:], px, 2, 1.0, 0.1, 0.1, *outs, None) == INVALID
    assert f(*bufs, None, 2, 1.0, 0.1, 0.1, *outs, None) == INVALID
    bad = (C.c_int64 * 2)(100, 0)
    assert f(*bufs, bad, 2, 1.0, 0.1, 0.1, *outs, None) == INVALID


def test_loss_ssim_rejects():
    f = lib().p2e_loss_ssim
    hw = (C.c_int32 * 2)(64, 64)
    args = dict(rgb=A, gt=A + 0x100000, hw=hw, nv=1, w=0.2, loss=A + 0x200000, d=A + 0x300000,
                scratch=A + 0x400000, sb=1 << 30)

    def call(**o):
        a = {**args, **o}
        return f(a["rgb"], a["gt"], a["hw"], a["nv"], a["w"], a["loss"], a["d"], a["scratch"], a["sb"], None)
    assert call(nv=0) == INVALID
    assert call(w=math.nan) == INVALID
    assert call(scratch=A + 64) == INVALID
    assert call(scratch=None) == INVALID
    assert call(sb=16) == INVALID
    assert call(hw=(C.c_int32 * 2)(0, 64)) == INVALID
    assert call(hw=(C.c_int32 * 2)(64, 9000)) == INVALID
    assert call(rgb=None) == INVALID


def test_loss_splat_area_rejects():
    f = lib().p2e_loss_splat_area
    assert f(A, A + 0x100000, 0, 0.1, A + 0x200000, A + 0x300000, None) == INVALID
    assert f(A, A + 0x100000, 100, -0.1, A + 0x200000, A + 0x300000, None) == INVALID
    assert f(A, A + 0x100000, 100, math.inf, A + 0x200000, A + 0x300000, None) == INVALID
    assert f(MIS, A + 0x100000, 100, 0.1, A + 0x200000, A + 0x300000, None) == INVALID
    assert f(A, A + 0x100000, 100, 0.1, None, A + 0x300000, None) == INVALID


def test_mlp_backward_and_adam_reject():
    g = gauss()
    f = lib().p2e_mlp_backward
    rest = [A + 0x1000000 + 0x100000 * k for k in range(6)]
    assert f(A, A + 0x100000, 0, A + 0x200000, C.byref(g), *rest, None) == INVALID
    assert f(A, A + 0x100000, 1000, MIS, C.byref(g), *rest, None) == INVALID
    assert f(A, A + 0x100000, 1000, None, C.byref(g), *rest, None) == INVALID
    assert f(A, A + 0x100000, 1000, A + 0x200000, None, *rest, None) == INVALID
    adam = lib().p2e_adam
    bufs = [A + 0x100000 * k for k in range(4)]
    assert adam(*bufs, _lib.MLP_PARAMS - 1, 1e-3, 0.9, 0.999, 1e-8, 1, A + 0x800000, None) == INVALID
    assert adam(*bufs, _lib.MLP_PARAMS, 1e-3, 0.9, 0.999, 1e-8, 0, A + 0x800000, None) == INVALID
    assert adam(None, *bufs[1:], _lib.MLP_PARAMS, 1e-3, 0.9, 0.999, 1e-8, 1, A + 0x800000, None) == INVALID


# ---------------------------------------------------------------- extras
def test_relight_rejects():
    f = lib().p2e_relight
    px = (C.c_int64 * 1)(128 * 128)
    light = (C.c_float * 4)(0.3, -0.5, 0.8, 1.0)
    planes = (A, A + 0x100000, A + 0x200000)
    out = A + 0x300000
    assert f(*planes, px, 0, light, 1, 0.2, None, out, None) == INVALID
    assert f(*planes, None, 1, light, 1, 0.2, None, out, None) == INVALID
    assert f(*planes, px, 1, None, 1, 0.2, None, out, None) == INVALID          # lights missing
    assert f(*planes, px, 1, light, _lib.P2E_MAX_LIGHTS + 1, 0.2, None, out, None) == INVALID
    assert f(*planes, px, 1, light, 1, math.nan, None, out, None) == INVALID
    zero = (C.c_float * 4)(0.0, 0.0, 0.0, 1.0)                                   # no direction
    assert f(*planes, px, 1, zero, 1, 0.2, None, out, None) == INVALID
    assert f(*planes, (C.c_int64 * 1)(-1), 1, light, 1, 0.2, None, out, None) == INVALID
    assert f(*planes, px, 1, light, 1, 0.2, (C.c_float * 3)(0, math.inf, 0), out, None) == INVALID
    assert f(None, *planes[1:], px, 1, light, 1, 0.2, None, out, None) == INVALID
    # no pixels at all: valid, nothing to do
    assert f(None, None, None, (C.c_int64 * 1)(0), 1, light, 1, 0.2, None, None, None) == OK


def test_point_raster_rejects():
    f = lib().p2e_point_raster
    z, o = A + 0x1000000, A + 0x2000000
    assert f(A, A + 0x100000, 100, None, 1, None, z, o, None, None) == INVALID
    assert f(A, A + 0x100000, 100, cams(), 0, None, z, o, None, None) == INVALID
    assert f(A, A + 0x100000, -1, cams(), 1, None, z, o, None, None) == INVALID
    assert f(A, A + 0x100000, 100, cams(width=0), 1, None, z, o, None, None) == INVALID
    assert f(A, A + 0x100000, 100, cams(cy=math.nan), 1, None, z, o, None, None) == INVALID
    assert f(A, A + 0x100000, 100, cams(), 1, (C.c_float * 3)(math.nan, 0, 0), z, o, None, None) == INVALID
    assert f(A, A + 0x100000, 100, cams(), 1, None, A + 4, o, None, None) == INVALID  # zbuf 8-byte words
    assert f(A, A + 0x100000, 100, cams(), 1, None, None, o, None, None) == INVALID
    assert f(MIS, A + 0x100000, 100, cams(), 1, None, z, o, None, None) == INVALID
    assert f(None, A + 0x100000, 100, cams(), 1, None, z, o, None, None) == INVALID


def test_kernel_probe_is_host_state_only():
    f = lib().p2e_set_kernel_probe
    pr = _lib.P2EKernelProbe(None, None, None)
    assert f(-1, C.byref(pr)) == INVALID
    assert f(4, C.byref(pr)) == INVALID
    for k in (_lib.P2E_PROBE_KNN, _lib.P2E_PROBE_BLEND, _lib.P2E_PROBE_MLP, _lib.P2E_PROBE_BLEND_BWD):
        assert f(k, C.byref(pr)) == OK       # attach (no events: nothing is recorded)
        assert f(k, None) == OK              # detach


def test_selftest_timeout_rejects():
    f = lib().p2e_selftest_timeout
    sb = _lib.SELFTEST_SCRATCH_BYTES
    assert f(5, 64, A, sb, A + 0x200000, None) == INVALID
    assert f(-1, 64, A, sb, A + 0x200000, None) == INVALID
    assert f(0, 0, A, sb, A + 0x200000, None) == INVALID         # a limit of zero rounds
    assert f(0, 1 << 30, A, sb, A + 0x200000, None) == INVALID   # above the library's own limit
    assert f(0, 64, A, sb - 1, A + 0x200000, None) == INVALID
    assert f(0, 64, A + 16, sb, A + 0x200000, None) == INVALID
    assert f(0, 64, A, sb, A + 0x200002, None) == INVALID
    assert f(0, 64, A, sb, None, None) == INVALID


def test_status_strings():
    names = {_lib.P2E_OK: "ok", _lib.P2E_ERR_INVALID_ARG: "invalid argument",
             _lib.P2E_ERR_CAPACITY: "key capacity exceeded", _lib.P2E_ERR_CUDA: "CUDA error",
             _lib.P2E_ERR_TIMEOUT: "device wait timed out", _lib.P2E_ERR_UNSUPPORTED: "unsupported"}
    for s, name in names.items():
        assert _lib.status_string(s) == name
    assert _lib.status_string(99) == "unknown status"

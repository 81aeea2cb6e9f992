"""The C-ABI library loads on a machine without a GPU and exports every
symbol include/p2e.h declares; host-side helpers answer without a device."""
import ctypes as C
import os
import re

import paper_2409_16504_gb300 as p2e
from paper_2409_16504_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "p2e.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(p2e_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    lib = p2e.load()
    syms = declared_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(_lib.EXPORTS)


def test_host_helpers_without_gpu():
    lib = p2e.load()
    c = lib.p2e_default_config()
    assert c.tile == 16 and abs(c.alpha_floor - 1 / 255) < 1e-9 and c.t_min > 0
    cams = p2e.render.make_cameras([dict(viewmat=[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 3]],
                                         fx=100, fy=100, cx=50, cy=40, width=100, height=80,
                                         near=0.01)])
    assert lib.p2e_total_tiles(cams, 1, 16) == 7 * 5
    assert lib.p2e_total_tiles(cams, 1, 12) == -1
    assert lib.p2e_scratch_bytes(0, 1000, 5000) > 0
    assert _lib.status_string(_lib.P2E_ERR_CAPACITY) == "key capacity exceeded"


def test_struct_layouts_match_header():
    # sizes of the POD structs as a C compiler lays them out
    assert C.sizeof(_lib.P2ECamera) == 4 * 12 + 4 * 4 + 4 * 2 + 4
    assert C.sizeof(_lib.P2EConfig) == 4 + 5 * 4 + 3 * 4 + 4
    assert C.sizeof(_lib.P2EGaussians) == 5 * 8 + 8
    assert C.sizeof(_lib.P2EBins) == 2 * 8 + 2 * 8 + 8 + 8 + 8 + 8 + 8 + 8 + 8 + 8
    assert C.sizeof(_lib.P2EKernelProbe) == 3 * 8

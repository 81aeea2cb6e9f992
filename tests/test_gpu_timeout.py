"""The bounded device waits give up, return and report P2E_ERR_TIMEOUT.

Every spin-wait of the library (the decoupled look-backs of the radix sort
and of the estimator's cell scan, the learned head's mbarrier waits, the
compositing's wait for deferred re-walks and its queue lock) has an
iteration limit.  p2e_selftest_timeout drives one of them into a wait that
can never be satisfied -- a predecessor tile that no CTA publishes, an
mbarrier arrival that never comes -- with a short limit.  The wait must
run out within milliseconds, the kernel must return, the status word must
read P2E_ERR_TIMEOUT (as p2e_bins_check reports it), and the GPU context
must stay usable: a render afterwards still matches the oracle.
"""
import ctypes as C
import time

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _selftest(which, spin_limit):
    from paper_2409_16504_gb300 import _lib
    from paper_2409_16504_gb300.render import P2EBins, _stream
    lib = _lib.load()
    scratch = torch.zeros(_lib.SELFTEST_SCRATCH_BYTES + 256, dtype=torch.uint8, device="cuda")
    sp = (scratch.data_ptr() + 255) & ~255
    words = torch.zeros(2, dtype=torch.int64, device="cuda")  # n_keys, status
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = lib.p2e_selftest_timeout(which, spin_limit, C.c_void_p(sp), _lib.SELFTEST_SCRATCH_BYTES,
                                  C.c_void_p(words.data_ptr() + 8), _stream())
    assert st == _lib.P2E_OK
    bins = P2EBins()
    bins.n_keys_dev = words.data_ptr()
    bins.status_dev = words.data_ptr() + 8
    bins.capacity = 0
    k = C.c_int64(-1)
    status = lib.p2e_bins_check(C.byref(bins), C.byref(k), _stream())  # synchronises
    return status, time.perf_counter() - t0


@pytest.mark.parametrize("which", [0, 1, 2, 3, 4])
def test_wait_gives_up_and_reports_timeout(which):
    from paper_2409_16504_gb300 import _lib
    status, dt = _selftest(which, 4096)
    assert status == _lib.P2E_ERR_TIMEOUT
    assert dt < 1.0, dt
    print(f"wait {which}: timed out after {dt * 1e3:.2f} ms")


def test_context_usable_after_timeouts():
    import oracle
    from gpu_common import cfg1_scene, gpu_render
    from paper_2409_16504_gb300 import _lib
    for which in (0, 1, 2, 3, 4):
        assert _selftest(which, 64)[0] == _lib.P2E_ERR_TIMEOUT
    g, cam = cfg1_scene()
    r, out = gpu_render(g, [cam])
    ref = oracle.render(g, cam)
    ok = ~ref["flag"]
    err = np.abs(out.view(0)["rgb"].cpu().numpy() - ref["rgb"])[:, ok].max()
    assert err <= 1e-4


def test_selftest_rejects_bad_arguments():
    from paper_2409_16504_gb300 import _lib
    lib = _lib.load()
    s = torch.zeros(_lib.SELFTEST_SCRATCH_BYTES + 256, dtype=torch.uint8, device="cuda")
    sp = C.c_void_p((s.data_ptr() + 255) & ~255)
    w = torch.zeros(1, dtype=torch.int32, device="cuda")
    wp = C.c_void_p(w.data_ptr())
    assert lib.p2e_selftest_timeout(5, 64, sp, _lib.SELFTEST_SCRATCH_BYTES, wp, None) == _lib.P2E_ERR_INVALID_ARG
    assert lib.p2e_selftest_timeout(0, 0, sp, _lib.SELFTEST_SCRATCH_BYTES, wp, None) == _lib.P2E_ERR_INVALID_ARG
    assert lib.p2e_selftest_timeout(0, 64, sp, 1024, wp, None) == _lib.P2E_ERR_INVALID_ARG

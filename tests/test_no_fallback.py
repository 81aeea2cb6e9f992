"""The package has no CPU fallback: without libp2e.so and without the CUDA
toolkit to build it, every entry of the public API raises instead of
computing anything.  Run in a fresh interpreter, so that the library this
test process may already have loaded is not the one asked for."""
import os
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = textwrap.dedent("""
    import os, shutil, sys, tempfile
    sys.path.insert(0, {root!r})
    import paper_2409_16504_gb300.build as b
    tmp = tempfile.mkdtemp()
    b.OUT = tmp
    b.LIB = os.path.join(tmp, "libp2e.so")          # not built
    shutil.which = lambda *a, **k: None             # no nvcc on PATH
    real_exists = os.path.exists
    os.path.exists = lambda p: False if str(p).endswith("nvcc") else real_exists(p)
    from paper_2409_16504_gb300 import _lib
    from paper_2409_16504_gb300.estimate import Estimator
    from paper_2409_16504_gb300 import render
    cams = [dict(viewmat=[[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 3]], fx=100, fy=100, cx=50, cy=40,
                 width=100, height=80, near=0.01)]
    results = []
    for name, call in [
        ("load", lambda: _lib.load()),
        ("Estimator", lambda: Estimator(1000, device="cpu")),
        ("Bins", lambda: render.Bins(1000, 35, 4096, device="cpu")),
        ("total_tiles", lambda: render.total_tiles(cams, 16)),
    ]:
        try:
            call()
            results.append(name + " ran")
        except RuntimeError as e:
            results.append(name + " raised: " + str(e).splitlines()[0])
    print("\\n".join(results))
""")


def test_public_api_raises_without_the_library():
    out = subprocess.run([sys.executable, "-c", PROBE.format(root=ROOT)], capture_output=True, text=True,
                         timeout=120, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = out.stdout.strip().splitlines()
    assert len(lines) == 4, lines
    for line in lines:
        assert "raised: nvcc not found: the CUDA toolkit is required to build libp2e" in line, lines

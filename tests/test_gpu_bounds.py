"""The bounds-checked build (-DPDEP_BOUNDS_CHECK, libpdep_check.so).

Its transform kernels test every index they read from the host-built sphere
tables (x-line members and columns, y-line slots) and report a failure
through the device status word instead of touching memory outside the
tables.  A child process with PDEP_BOUNDS_CHECK=1 runs the calls of
checked_calls.py (every supported grid shape, a mixed PDEP solve, chi0bar
applications, Lanczos chains) through that library: no index may fail its
test, and the results must equal those of the normal library in this
process: the transforms to rounding (1e-14 FP64, 1e-6 FP32; a skipped
access would change them at order one), the solves, which accumulate sums
with atomics in a run-dependent order, to their accuracy (1e-10 FP64, 1e-8
for the mixed path, whose FP32 inner iterations diverge at FP32 rounding
before the FP64 refinement brings both to the same tolerance).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_common import lib_ready, need_gpu, rel

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_checked_build_agrees(tmp_path):
    need_gpu()
    lib_ready()
    from paper_1501_03141_gb300 import build
    build.build(bounds_check=True)
    path = tmp_path / "checked.npz"
    env = dict(os.environ, PDEP_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_calls.py"), str(path)],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    got = dict(np.load(path))
    assert int(got["bounds_checked"]) == 1

    import checked_calls
    ref = checked_calls.run_calls()
    assert int(ref["bounds_checked"]) == 0
    assert sorted(got) == sorted(ref)
    for k, v in ref.items():
        if k == "bounds_checked":
            continue
        if k.startswith(("grid_", "h64_")):
            assert rel(got[k], v) < 1e-14, k
        elif k.startswith("h32_"):
            assert rel(got[k], v) < 1e-6, k
        elif k in ("tiny_eig", "cube48_chi0"):
            # mixed path: the FP32 inner CG's reductions run in a different
            # order, both results meet the 1e-10 Sternheimer tolerance
            assert rel(got[k], v) < 1e-8, k
        else:
            assert rel(got[k], v) < 1e-10, k

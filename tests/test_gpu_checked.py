"""The bounds-checked build and injected allocation failures on the GPU.

* libaf_checked.so (AF_CHECKED=1) runs integration, the bit view, scoring on
  the fast and the bounds-checked paths, the point layer and a batched tick
  bit for bit like the oracle and the plain library, and no bounds check
  fails (tests/checked_run.py, in a child process: the binding loads one
  library per process).
* af_create with an allocation failure injected at every position returns
  AF_ERR_CUDA and releases what it had allocated: the device's free memory
  after the failures equals what it was before them."""
import os
import subprocess
import sys

import pytest

from paper_2608_06412_gb300 import af, workload

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_matches_and_no_check_fails():
    af.load()  # builds both libraries if stale
    env = dict(os.environ, AF_CHECKED="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_run.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "CHECKED OK" in r.stdout


def test_injected_allocation_failures_release_everything():
    import ctypes as C
    import torch
    lib = af.load()
    torch.cuda.set_device(0)
    torch.cuda.synchronize()
    cc = workload.single_frame().af_config(hash_capacity=1 << 20, pool_blocks=1 << 16,
                                           max_returns=1 << 16, max_points=1 << 16)._c()
    free0, _ = torch.cuda.mem_get_info()
    failures = 0
    for k in range(64):
        h = C.c_void_p()
        os.environ["AF_FAIL_ALLOC_AT"] = str(k)
        try:
            st = lib.af_create(C.byref(cc), C.byref(h))
        finally:
            del os.environ["AF_FAIL_ALLOC_AT"]
        if st == af.OK:                       # k is past af_create's last allocation
            assert lib.af_destroy(h) == af.OK
            break
        assert st == af.ERR_CUDA and not h.value
        assert f"injected failure at allocation {k}".encode() in lib.af_last_error(None)
        failures += 1
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert failures >= 10
    assert abs(free1 - free0) <= 64 << 20, (free0, free1)

"""The C ABI without a GPU: libaf loads, exports every symbol that
include/af.h declares, and its host-only kernel rasteriser produces exactly
the oracle's integer kernels (the two are written independently)."""
import os
import re

import numpy as np
import pytest

import oracle
from paper_2608_06412_gb300 import af, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(af_[a-z_0-9]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    lib = af.load()
    declared = _declared()
    assert declared, "no declarations found"
    assert declared == set(af.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name
    assert b"sm_103a" in lib.af_version()


def test_host_errors_are_reported_without_gpu():
    lib = af.load()
    t = af.ToolConfig(radius=-1.0, length=0.25, self_excl=0.04, corr_radius=0.05,
                      corr_length=1.0)
    with pytest.raises(af.AfError) as e:
        af.kernel_offsets(t, 0.02, [0, 0, 1], af.KERNEL_TOOL)
    assert e.value.status == 1
    assert lib.af_create(None, None) == 1


def test_checked_build_exports_the_same_symbols():
    """libaf_checked.so (the bounds-checked build) exports every declared
    entry point and names itself in af_version."""
    import ctypes as C
    from paper_2608_06412_gb300 import build as B
    af.load()
    lib = C.CDLL(B.LIB_CHECKED)
    for name in _declared():
        assert hasattr(lib, name), name
    lib.af_version.restype = C.c_char_p
    assert b"checked" in lib.af_version() and b"checked" not in af.load().af_version()


def test_injected_allocation_failure():
    """AF_FAIL_ALLOC_AT=0 makes af_create's first device allocation fail:
    AF_ERR_CUDA, nothing returned, the injection named in the message. The
    check comes before the allocation, so no GPU is needed."""
    import ctypes as C
    from paper_2608_06412_gb300 import workload
    lib = af.load()
    cc = workload.single_frame().af_config()._c()
    h = C.c_void_p(123)
    os.environ["AF_FAIL_ALLOC_AT"] = "0"
    try:
        st = lib.af_create(C.byref(cc), C.byref(h))
    finally:
        del os.environ["AF_FAIL_ALLOC_AT"]
    assert st == af.ERR_CUDA and not h.value
    assert b"injected failure at allocation 0" in lib.af_last_error(None)


def test_noalloc_rejects_boxes_beyond_its_limit():
    """af_integrate_scan_noalloc rejects a box of more than 2^40 voxels before
    touching the GPU, including boxes whose voxel count would wrap a 64-bit
    product (2^23 per axis = 2^69 voxels)."""
    import ctypes as C
    from paper_2608_06412_gb300 import workload
    lib = af.load()
    cc = workload.single_frame().af_config()._c()
    pose = np.eye(4, dtype=np.float32).reshape(16)
    bmin = np.zeros(3, np.int32)
    dummy = C.c_void_p(256)  # never dereferenced: the call returns before any CUDA work
    for dims in ((1 << 23, 1 << 23, 1 << 23), (1 << 20, 1 << 20, 2), (1 << 23, 1 << 23, 1 << 8)):
        bdim = np.asarray(dims, np.uint32)
        st = lib.af_integrate_scan_noalloc(C.byref(cc), C.c_void_p(0), 0, af._np_ptr(pose),
                                           af._np_ptr(bmin), af._np_ptr(bdim), dummy, dummy,
                                           C.c_void_p(0))
        assert st == 1, dims
        assert b"2^40" in lib.af_last_error(None)


def _tools():
    yield synth.SINGLE_FRAME["tool"], 0.02
    yield dict(radius=0.03, length=0.15, self_excl=0.005, corr_radius=0.03,
               corr_length=0.5, cos_theta_max=0.0, n_c=5, strict=0), 0.01
    yield dict(radius=0.06, length=0.40, self_excl=0.06, corr_radius=0.06,
               corr_length=0.3, cos_theta_max=0.342, n_c=5, strict=1), 0.02


@pytest.mark.parametrize("ti", [0, 1, 2])
def test_kernel_tables_match_oracle(ti):
    """The library and the oracle rasterise every kernel to the same integer
    set, for a Fibonacci direction set and the axis directions (exact ties)."""
    tool, v = list(_tools())[ti]
    dirs = np.concatenate([synth.fibonacci_dirs(24),
                           np.array([[0, 0, 1], [1, 0, 0], [0, -1, 0]], np.float32)])
    ot = oracle.Tool(**tool)
    at = af.ToolConfig(**tool)
    for u in dirs:
        for which in (0, 1):
            a = af.kernel_offsets(at, v, u, which)
            o = oracle.kernel_offsets(ot, v, u, which)
            o = o[np.lexsort((o[:, 0], o[:, 1], o[:, 2]))]
            np.testing.assert_array_equal(a, o)
        np.testing.assert_array_equal(af.arm_offsets(v, 0.06, u), oracle.arm_offsets(v, 0.06, u))

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

"""Builds libaf.so (the sm_103a CUDA library behind include/af.h) in-tree,
and its bounds-checked twin libaf_checked.so (the same sources compiled with
AF_CHECKED: every pool, plane-word and run-table index of the integration,
bit-view and scoring kernels is checked and a failure latches AF_ERR_CHECK).

Each translation unit of both builds is compiled in parallel with nvcc, then
linked into ``paper_2608_06412_gb300/libaf.so`` and ``libaf_checked.so``.
Floating-point contraction is off on both the device (--fmad=false) and the
host (-ffp-contract=off) side: the integer results of the method are decided
by single-precision arithmetic that must round exactly as written.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libaf.so")
LIB_CHECKED = os.path.join(PKG, "libaf_checked.so")
BUILD_DIR = os.path.join(PKG, "_build")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libaf")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(LIB_CHECKED):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_CHECKED))
    return any(os.path.getmtime(d) > t for d in _deps())


def flags() -> list:
    return ["-O3", "-std=c++17", ARCH, "-lineinfo", "--fmad=false",
            "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math",
            "-I", INCLUDE, "-I", CSRC]


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libaf.so and libaf_checked.so if any source is newer than
    them; return the path of libaf.so."""
    if not force and not _stale():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    procs = []
    objs = {LIB: [], LIB_CHECKED: []}
    for lib, extra, tag in ((LIB, [], ""), (LIB_CHECKED, ["-DAF_CHECKED"], ".checked")):
        for src in _sources():
            obj = os.path.join(BUILD_DIR, os.path.basename(src) + tag + ".o")
            objs[lib].append(obj)
            cmd = [nvcc, *flags(), *extra, "-c", src, "-o", obj]
            if verbose and not extra:
                cmd.insert(1, "-Xptxas=-v")
            procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                stderr=subprocess.STDOUT, text=True)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stderr.write(out)
        if p.returncode != 0:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    for lib, o in objs.items():
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run([nvcc, ARCH, "-shared", "-o", tmp, *o], check=True)
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

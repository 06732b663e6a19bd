"""Compile the CUDA library (sm_103a) in-tree: paper_1108_5561_gb300/_build/librlb.so."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "librlb.so")
# the same library with the device-side range and finiteness checks (RLB_CHECKS)
LIB_CHECKED = os.path.join(OUT_DIR, "librlb_checked.so")
SOURCES = ["rlb_api.cu", "rlb_host.cpp"]
HEADERS = ["rlb_kernels.cuh", "rlb_stage_x2.cuh", "rlb_stage_mp.cuh", "rlb_stage_mpt.cuh", "rlb_peaks.cuh", "rlb_adjoint.cuh", "rlb_host.hpp", os.path.join("..", "..", "include", "rlb.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(os.path.join(CSRC, f)) > t for f in SOURCES + HEADERS)


def _command(lib: str, checked: bool, verbose: bool):
    cmd = [nvcc(), "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-shared",
           "-o", lib] + [os.path.join(CSRC, s) for s in SOURCES]
    if checked:
        cmd.insert(1, "-DRLB_CHECKS=1")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    return cmd


def build(force: bool = False, verbose: bool = False, checked: bool = False, both: bool = False) -> str:
    """Compile the library (checked=True: the RLB_CHECKS build; both=True: the
    two builds side by side).  Returns the path of the (first) library."""
    want = [(LIB, False), (LIB_CHECKED, True)] if both else [(LIB_CHECKED if checked else LIB, checked)]
    todo = [(lib, c) for lib, c in want if force or _stale(lib)]
    if todo:
        os.makedirs(OUT_DIR, exist_ok=True)
        procs = []
        for lib, c in todo:
            tmp = lib + ".tmp%d" % os.getpid()
            procs.append((subprocess.Popen(_command(tmp, c, verbose)), tmp, lib))
        failed = [p for p, _, _ in procs if p.wait() != 0]
        if failed:
            raise subprocess.CalledProcessError(failed[0].returncode, failed[0].args)
        for _, tmp, lib in procs:
            os.replace(tmp, lib)
    return want[0][0]


if __name__ == "__main__":
    print(build(force=True, verbose=True))

"""Build the CUDA library libep.so in-tree for sm_103a (nvcc, no torch types).

Usage: python -m paper_2302_12519_gb300.build [--force] [--verbose-ptxas]
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libep.so")
SOURCES = [os.path.join(CSRC, "ep_api.cu"), os.path.join(CSRC, "ep_sdf.cu")]
HEADERS = [os.path.join(CSRC, h) for h in ("ep_kernels.cuh", "ep_common.cuh", "ep_stencil.cuh", "ep_aux.cuh")]
DEPS = SOURCES + HEADERS + [os.path.join(ROOT, "include", h) for h in ("ep.h", "ep_sdf.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in DEPS)


def build(force: bool = False, ptxas_verbose: bool = False, defines=None, out: str = None) -> str:
    """Compile libep.so.  ``defines`` (e.g. {"EP_WARPS": 8}) override the tile
    constants; ``out`` writes the library elsewhere (used for tuning builds)."""
    target = out or LIB
    if out is None and not defines and not force and not needs_build():
        return LIB
    tmp = target + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "--threads", "2",
           "-I", os.path.join(ROOT, "include"), "-o", tmp, *SOURCES]
    for k, v in (defines or {}).items():
        cmd.insert(1, f"-D{k}={v}")
    if ptxas_verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, cwd=HERE, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed building libep.so")
    if ptxas_verbose:
        sys.stderr.write(r.stderr)
    os.replace(tmp, target)
    return target


if __name__ == "__main__":
    build(force="--force" in sys.argv, ptxas_verbose="--verbose-ptxas" in sys.argv)
    print(LIB)

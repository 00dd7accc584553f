"""Compile libzig_gb300.so in-tree with nvcc for sm_103a (GB300).

    python -m paper_2405_19493_gb300.build [--force] [-v]

The library is csrc/zig_lib.cu (kernels and the C ABI) and csrc/zig_server.cpp
(the mutation service's scheduler), plus their headers; the
output goes to paper_2405_19493_gb300/_lib/libzig_gb300_<arch>.so (git-ignored),
named by the host architecture because the x86 build host and the aarch64 GPU
host share the tree.
"""

from __future__ import annotations

import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB_DIR = os.path.join(HERE, "_lib")
SOURCES = ["zig_lib.cu", "zig_server.cpp"]
DEPS = ["zig_lib.cu", "zig_server.cpp", "zig_device.cuh", "z128_batch.cuh", "z256_batch.cuh", "zig_tables.inc"]
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]


def lib_path() -> str:
    return os.path.join(LIB_DIR, f"libzig_gb300_{platform.machine()}.so")


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libzig_gb300")
    return cand


def _stale(out: str) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    deps = [os.path.join(CSRC, d) for d in DEPS] + [os.path.join(INCLUDE, "zig.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    out = lib_path()
    if not force and not _stale(out):
        return out
    os.makedirs(LIB_DIR, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-O3", "-std=c++17", *ARCH_FLAGS, "-lineinfo", "-shared",
           "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread", "-cudart", "shared", "-I", INCLUDE,
           "-o", tmp] + [os.path.join(CSRC, s) for s in SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    p = build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(p)

"""Compile the CUDA library in-tree: ``_build/libfitspots.so`` for sm_103a.

nvcc cross-compiles without a GPU; the build is skipped when the library is newer than
every source it depends on.
"""
from __future__ import annotations

import os
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
SOURCES = [PKG / "csrc" / "fitspots.cu", PKG / "csrc" / "backward.cu", PKG / "csrc" / "serving.cu",
           PKG / "csrc" / "start.cu", PKG / "csrc" / "explicit.cu",
           PKG / "csrc" / "weighted.cu"]
HEADERS = [ROOT / "include" / "fitspots.h"]
LIB = PKG / "_build" / "libfitspots.so"
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> Path:
    LIB.parent.mkdir(exist_ok=True)
    newest = max(p.stat().st_mtime for p in SOURCES + HEADERS)
    if not force and LIB.exists() and LIB.stat().st_mtime >= newest:
        return LIB
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
    # no -split-compile: it made register allocation vary from build to build, with spills
    cmd = [nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           f"-I{ROOT / 'include'}", "-o", str(tmp)] + [str(s) for s in SOURCES]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))

"""Compile the CUDA library in-tree: ``_build/libfitspots.so`` for sm_103a.

nvcc cross-compiles without a GPU. Every translation unit is compiled to an object file of
its own, in parallel, then linked once; a unit is recompiled only when it or the C header is
newer than its object.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
SOURCES = [CSRC / n for n in ("fitspots.cu", "backward.cu", "serving.cu", "start.cu",
                              "explicit.cu", "weighted.cu", "poisson.cu", "background.cu",
                              "probe.cu")]
HEADERS = [ROOT / "include" / "fitspots.h", CSRC / "warp_lm.cuh"]
BUILD = PKG / "_build"
LIB = BUILD / "libfitspots.so"
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
# no -split-compile: it made register allocation vary from build to build, with spills
FLAGS = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _compile(src: Path, verbose: bool) -> Path:
    obj = BUILD / (src.stem + ".o")
    newest = max(p.stat().st_mtime for p in [src] + HEADERS)
    if obj.exists() and obj.stat().st_mtime >= newest:
        return obj
    tmp = obj.with_suffix(f".{os.getpid()}.tmp.o")
    cmd = [nvcc(), *FLAGS, f"-I{ROOT / 'include'}", "-c", str(src), "-o", str(tmp)]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(tmp, obj)
    return obj


def build(force: bool = False, verbose: bool = False) -> Path:
    BUILD.mkdir(exist_ok=True)
    if force:
        for src in SOURCES:
            (BUILD / (src.stem + ".o")).unlink(missing_ok=True)
    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), SOURCES))
    if LIB.exists() and LIB.stat().st_mtime >= max(o.stat().st_mtime for o in objs):
        return LIB
    tmp = LIB.with_suffix(f".{os.getpid()}.tmp")
    subprocess.run([nvcc(), ARCH, "-shared", "-o", str(tmp)] + [str(o) for o in objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))

"""Build libpbcg.so (the sm_103a CUDA library) in-tree with nvcc.

    python -m paper_2404_13216_gb300.build        # or build_library() from Python

Output: paper_2404_13216_gb300/_build/libpbcg.so, and with checked=True
libpbcg_checked.so, the same library with device-side bounds checks
(PBCG_CHECKS=1).  Device code is compiled with -fmad=false so that the only
fused multiply-adds are the explicit __fma_rn calls of the fixed rounding
forms.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC_DIR = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libpbcg.so")
LIB_CHECKED = os.path.join(OUT_DIR, "libpbcg_checked.so")
SOURCES = ["api.cu", "noalloc.cu"]
HEADERS = ["exdot.cuh", "kernels.cuh", "tma.cuh", "batched.cuh", "cluster.cuh", "dist.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(SRC_DIR, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "pbcg.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(lib: str, extra: list, verbose: bool) -> list:
    """Start one nvcc per translation unit for `lib`; returns (objs, procs)."""
    flags = [ARCH, "-O3", "-lineinfo", "-fmad=false", "-std=c++17", "-Xcompiler", "-fPIC"] + extra
    if verbose:
        flags.append("-Xptxas=-v")
    tag = os.path.basename(lib).replace(".so", "")
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, src.replace(".cu", f".{tag}.{os.getpid()}.o"))
        objs.append(obj)
        procs.append(subprocess.Popen([_nvcc()] + flags + ["-c", os.path.join(SRC_DIR, src), "-o", obj],
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    return objs, procs


def _link(lib: str, objs: list, procs: list, verbose: bool) -> None:
    errs = []
    for p in procs:
        out, err = p.communicate()
        if p.returncode != 0:
            errs.append(out + err)
        elif verbose:
            sys.stderr.write(err)
    if errs:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    tmp = lib + f".tmp{os.getpid()}"
    r = subprocess.run([_nvcc(), ARCH, "-shared", "-o", tmp] + objs + ["-ldl"], capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib)


def build_library(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build libpbcg.so (and, with checked=True, also libpbcg_checked.so, the
    translation units of both compiled in parallel); returns libpbcg.so."""
    jobs = [(LIB, [])] + ([(LIB_CHECKED, ["-DPBCG_CHECKS=1"])] if checked else [])
    jobs = [(lib, extra) for lib, extra in jobs if force or _stale(lib)]
    if not jobs:
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    started = [(lib, *_compile(lib, extra, verbose)) for lib, extra in jobs]
    for lib, objs, procs in started:
        _link(lib, objs, procs, verbose)
    return LIB


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose="-v" in sys.argv, checked=True))

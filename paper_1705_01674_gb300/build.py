"""Builds libsgwls.so in-tree with nvcc for sm_103a (GB300).

Each translation unit under csrc/ is compiled in parallel, then linked into
``paper_1705_01674_gb300/libsgwls.so``.  Objects go to ``_build/`` next to
this file.  A TU is rebuilt only when it or a header is newer than its
object.  Usage: ``python -m paper_1705_01674_gb300.build [--force]``.

Development shortcut: with ``SGWLS_RADII=1,2`` only those radii are
compiled; the launchers of the other radii are built as stubs that return
"unsupported".  The default (unset) builds every radius.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libsgwls.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "--expt-relaxed-constexpr",
           "-I", INCLUDE]


def _nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found")
    return cand


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _radius_of(src: str):
    base = os.path.basename(src)
    if base.startswith("sgwls_r") and base[7:-3].isdigit():
        return int(base[7:-3])
    return None


def _compile(src: str, force: bool, extra) -> str:
    radii = os.environ.get("SGWLS_RADII")
    r = _radius_of(src)
    stub = bool(radii) and r is not None and str(r) not in radii.split(",")
    tag = ".stub.o" if stub else ".o"
    obj = os.path.join(BUILD, os.path.basename(src).replace(".cu", tag))
    if stub:
        extra = list(extra) + ["-DSGWLS_STUB_RADIUS"]
    if not force and os.path.exists(obj):
        newest = max(os.path.getmtime(p) for p in [src] + _headers())
        if os.path.getmtime(obj) >= newest:
            return obj
    cmd = [_nvcc(), *ARCH, *NVFLAGS, *extra, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    workers = max(1, min(len(srcs), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(lambda s: _compile(s, force, list(extra)), srcs))
    if True:  # linking is cheap; relink so stub/full object sets never mix up
        cmd = [_nvcc(), *ARCH, "-shared", "-o", LIB, *objs, "-lcudart_static", "-lrt", "-lpthread", "-ldl"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)

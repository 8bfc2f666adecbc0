"""Builds libsgwls.so in-tree with nvcc for sm_103a (GB300).

Translation units: ``csrc/sgwls_api.cu``, ``csrc/sgwls_noalloc.cu`` and
``csrc/sgwls_inst.cu`` compiled once per (radius 1..8, channel group 1..4)
pair with ``-DSGWLS_R`` / ``-DSGWLS_CC`` (the kernels of one pair per object,
so the 34 compilations run in parallel), then linked into
``paper_1705_01674_gb300/libsgwls.so``.  Objects go to ``_build/`` next to
this file; an object is rebuilt only when its source or a header is newer.
Usage: ``python -m paper_1705_01674_gb300.build [--force]``.

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


RADII = range(1, 9)
GROUPS = range(1, 5)


def _units():
    """(source, object base name, extra flags, radius or None) of every TU."""
    units = [(os.path.join(CSRC, "sgwls_api.cu"), "sgwls_api", [], None),
             (os.path.join(CSRC, "sgwls_noalloc.cu"), "sgwls_noalloc", [], None)]
    inst = os.path.join(CSRC, "sgwls_inst.cu")
    for r in RADII:
        for cc in GROUPS:
            units.append((inst, f"sgwls_inst_r{r}_c{cc}", [f"-DSGWLS_R={r}", f"-DSGWLS_CC={cc}"], r))
    # the backward's widest group at r = 1: u and v of three channels
    units.append((inst, "sgwls_inst_r1_c6", ["-DSGWLS_R=1", "-DSGWLS_CC=6"], 1))
    return units


def _compile(unit, force: bool, extra) -> str:
    src, name, flags, r = unit
    radii = os.environ.get("SGWLS_RADII")
    stub = bool(radii) and r is not None and str(r) not in radii.split(",")
    obj = os.path.join(BUILD, name + (".stub.o" if stub else ".o"))
    flags = list(flags) + list(extra) + (["-DSGWLS_STUB_RADIUS"] if stub else [])
    if not force and os.path.exists(obj):
        newest = max(os.path.getmtime(p) for p in [src] + _headers())
        if os.path.getmtime(obj) >= newest:
            return obj
    cmd = [_nvcc(), *ARCH, *NVFLAGS, *flags, "-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed for {name}:\n{res.stdout}\n{res.stderr}")
    return obj


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    units = _units()
    # the large radii compile longest: start them first
    order = sorted(units, key=lambda u: -(u[3] or 0))
    workers = max(1, min(len(units), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(workers) as ex:
        done = dict(zip([u[1] for u in order], ex.map(lambda u: _compile(u, force, list(extra)), order)))
    objs = [done[u[1]] for u in units]
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

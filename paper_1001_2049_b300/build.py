"""Build libvr.so in-tree with nvcc for sm_103a (B300).

``python -m paper_1001_2049_b300.build [--force] [--ptxas-info]``

Every source is compiled to its own object in parallel (the texture kernels
are split by storage format so their instantiations compile side by side),
then the objects are linked into ``libvr.so`` next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(PKG, "libvr.so")
OBJ = os.path.join(PKG, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvr")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _inputs():
    return (sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(INCLUDE, "*.h")))


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def _flags(ptxas_info: bool):
    f = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "-I", INCLUDE, "-I", CSRC]
    if ptxas_info:
        f.insert(0, "-Xptxas=-v")
    extra = os.environ.get("VR_NVCC_EXTRA", "").split()
    return extra + f                   # e.g. -DVR_BATCH_MIN_BLOCKS=3 for tuning builds


def _compile(src, flags):
    obj = os.path.join(OBJ, os.path.basename(src) + ".%d.o" % os.getpid())
    res = subprocess.run([nvcc(), *flags, "-c", "-o", obj, src], capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, res.stdout, res.stderr))
    return obj, res.stderr


def build(force: bool = False, ptxas_info: bool = False, verbose: bool = False) -> str:
    """Compile every CUDA/C++ source of the package into libvr.so."""
    if not force and not ptxas_info and not stale():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    flags = _flags(ptxas_info)
    srcs = sources()
    if verbose:
        print(" ".join([nvcc(), *flags, "-c", "<src>"]), file=sys.stderr)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        results = list(ex.map(lambda s: _compile(s, flags), srcs))
    objs = [o for o, _ in results]
    if ptxas_info:
        for src, (_, err) in zip(srcs, results):
            sys.stderr.write("== %s\n%s" % (os.path.basename(src), err))
    tmp = LIB + ".tmp%d" % os.getpid()
    res = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True,
                         text=True)
    for o in objs:
        os.remove(o)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n" + res.stdout + res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, ptxas_info="--ptxas-info" in sys.argv, verbose=True)
    print(LIB)

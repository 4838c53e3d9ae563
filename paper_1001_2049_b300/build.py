"""Build libvr.so in-tree with nvcc for sm_103a (B300).

``python -m paper_1001_2049_b300.build [--force] [--ptxas-info] [--debug]``

Every source is compiled to its own object in parallel (the texture kernels
are split by storage format so their instantiations compile side by side),
then the objects are linked into ``libvr.so`` next to this file.  ``--debug``
builds the checked library ``libvr_debug.so`` instead (VR_DEBUG: the kernels
test the indices they compute and record failures for vr_debug_status).
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
DEBUG_LIB = os.path.join(PKG, "libvr_debug.so")
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


def stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _inputs())


def _flags(ptxas_info: bool, debug: bool = False):
    f = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O3",
         "-I", INCLUDE, "-I", CSRC]
    if debug:
        f.append("-DVR_DEBUG")
    if ptxas_info:
        f.insert(0, "-Xptxas=-v")
    extra = os.environ.get("VR_NVCC_EXTRA", "").split()
    return extra + f                   # e.g. -DVR_BATCH_MIN_BLOCKS=3 for tuning builds


def _compile(src, flags):
    tag = ".dbg" if "-DVR_DEBUG" in flags else ""
    obj = os.path.join(OBJ, os.path.basename(src) + tag + ".%d.o" % os.getpid())
    res = subprocess.run([nvcc(), *flags, "-c", "-o", obj, src], capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, res.stdout, res.stderr))
    return obj, res.stderr


def build(force: bool = False, ptxas_info: bool = False, verbose: bool = False,
          debug: bool = False) -> str:
    """Compile every CUDA/C++ source of the package into libvr.so (the
    checked libvr_debug.so with debug=True)."""
    lib = DEBUG_LIB if debug else LIB
    if not force and not ptxas_info and not stale(lib):
        return lib
    os.makedirs(OBJ, exist_ok=True)
    flags = _flags(ptxas_info, debug)
    srcs = sources()
    if verbose:
        print(" ".join([nvcc(), *flags, "-c", "<src>"]), file=sys.stderr)
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        results = list(ex.map(lambda s: _compile(s, flags), srcs))
    objs = [o for o, _ in results]
    if ptxas_info:
        for src, (_, err) in zip(srcs, results):
            sys.stderr.write("== %s\n%s" % (os.path.basename(src), err))
    tmp = lib + ".tmp%d" % os.getpid()
    res = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True,
                         text=True)
    for o in objs:
        os.remove(o)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n" + res.stdout + res.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, ptxas_info="--ptxas-info" in sys.argv,
                verbose=True, debug="--debug" in sys.argv))

"""Build libmmba.so (the CUDA library) in-tree for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into one shared library next to this file.  Re-running only rebuilds
what changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmmba.so")
CHECKED_LIB = os.path.join(HERE, "libmmba_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + os.path.join(ROOT, "include")]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found (CUDA toolkit required to build libmmba)")
    return cand


def _deps():
    return (glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
            glob.glob(os.path.join(ROOT, "include", "*.h")))


def _compile(src: str, extra: list[str], obj_dir: str = OBJ) -> str:
    obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
    newest_dep = max([os.path.getmtime(src)] + [os.path.getmtime(d) for d in _deps()])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest_dep:
        return obj
    tmp = obj + f".tmp{os.getpid()}"
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, obj)
    return obj


def build(verbose_ptxas: bool = False, force: bool = False, checked: bool = False) -> str:
    """Compile every .cu under csrc/ and link libmmba.so; returns its path.
    checked=True builds libmmba_checked.so instead: the same library with the
    kernels' index checks compiled in (a stand-in for a memory sanitizer)."""
    obj_dir = OBJ + ("_checked" if checked else "")
    lib = CHECKED_LIB if checked else LIB
    os.makedirs(obj_dir, exist_ok=True)
    if force:
        for f in glob.glob(os.path.join(obj_dir, "*.o")):
            os.remove(f)
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    extra = (["-Xptxas", "-v"] if verbose_ptxas else []) + (["-DMMBA_CHECKED"] if checked else [])
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, obj_dir), srcs))
    if (not os.path.exists(lib)) or max(os.path.getmtime(o) for o in objs) > os.path.getmtime(lib):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build())

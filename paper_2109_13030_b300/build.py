"""Builds libtrajam.so (the C-ABI library) in-tree for sm_103a with nvcc."""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libtrajam.so")
# the debug build: the fused kernels bounds-check their array indices and
# report an out-of-bounds index in the status word instead of trapping
LIB_DEBUG = os.path.join(HERE, "libtrajam_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _headers() -> list[str]:
    return (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + [os.path.join(ROOT, "include", "trajam.h")])


def _newer(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(p) > t for p in deps)


def _stale(lib: str) -> bool:
    return _newer(lib, sources() + _headers())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          debug: bool = False) -> str:
    """Compiles every source to an object of its own (in parallel, under
    _build/, recompiling only sources newer than their object) and links
    the shared library."""
    lib = LIB_DEBUG if debug else LIB
    if not force and not _stale(lib):
        return lib
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
             "-Xcompiler", "-fvisibility=hidden", "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    if extra:
        flags[0:0] = extra
    if debug:
        flags.insert(0, "-DAM_DEBUG_BOUNDS")
    objdir = os.path.join(ROOT, "_build", "debug" if debug else "release")
    os.makedirs(objdir, exist_ok=True)
    headers = _headers()
    jobs = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        if force or extra or _newer(obj, [src, *headers, os.path.abspath(__file__)]):
            jobs.append((src, obj))

    def compile_one(job):
        src, obj = job
        subprocess.check_call([nvcc, *flags, "-c", src, "-o", obj + ".tmp"])
        os.replace(obj + ".tmp", obj)

    with ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        list(ex.map(compile_one, jobs))
    objs = [os.path.join(objdir, os.path.basename(s) + ".o") for s in sources()]
    subprocess.check_call([nvcc, *ARCH, "-shared", "-o", lib + ".tmp", *objs, "-lcudart"])
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv, debug="--debug" in sys.argv))

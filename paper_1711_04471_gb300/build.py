"""Build libgbsw.so (the CUDA library behind include/gbsw.h) for sm_103a.

Each translation unit under csrc/ is compiled in parallel with nvcc and the
objects are linked into paper_1711_04471_gb300/libgbsw.so.  No cmake; a
rebuild happens only when a source or header is newer than the library.
build(debug=True) makes the bounds-checked variant libgbsw_debug.so from
the same sources (GBSW_DEBUG_BOUNDS=1, objects in _build_debug/).
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgbsw.so")
OBJDIR_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libgbsw_debug.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgbsw.so")


def _flags(verbose: bool):
    f = [ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I" + os.path.join(ROOT, "include"),
         "--expt-relaxed-constexpr"]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = glob.glob(os.path.join(CSRC, "*")) + glob.glob(os.path.join(ROOT, "include", "*.h")) + [__file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Path of libgbsw.so (of libgbsw_debug.so with debug), compiled first
    if a source is newer.  With GBSW_DEBUG_BOUNDS=1 in the environment the
    product build also brings the debug library up to date (it is the one
    the binding then loads)."""
    if not debug and os.environ.get("GBSW_DEBUG_BOUNDS") == "1":
        build(force, verbose, debug=True)
    lib, objdir = (LIB_DEBUG, OBJDIR_DEBUG) if debug else (LIB, OBJDIR)
    if not force and not _stale(lib):
        return lib
    os.makedirs(objdir, exist_ok=True)
    cc = nvcc()
    srcs = sources()
    extra = ["-DGBSW_DEBUG_BOUNDS=1"] if debug else []

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src) + ".o")
        cmd = [cc, *_flags(verbose), *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 or verbose:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, ARCH, "-shared", "-o", tmp, *objs, "-lcudart", "-lcuda"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))

"""Compile the FP64 CPU oracle (plain C) into oracle/liboracle.so, and the
same sources with OpenMP into oracle/liboracle_omp.so.

Test infrastructure: only tests, the smoke check and the bench's CPU-baseline
leg load the result.  -ffp-contract=off keeps every FP64 operation rounded
as written (no fused multiply-add), so the oracle is reproducible across
x86-64 and aarch64 hosts.  The OpenMP build runs the outer loop of each
per-cell map on all host cores and keeps every sum serial; it exists to
time the oracle on all cores and gives bitwise the same results.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["sw_oracle.c", "les_oracle.c", "unet_oracle.c"]
LIB = os.path.join(HERE, "liboracle.so")
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")


def _build_one(out: str, extra, force: bool) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    if not force and os.path.exists(out):
        mtime = os.path.getmtime(out)
        if all(os.path.getmtime(s) <= mtime for s in srcs + [__file__]):
            return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", *extra,
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False, openmp: bool = False) -> str:
    """Path of the serial library (openmp=False) or of the OpenMP one,
    compiled first if a source is newer."""
    if openmp:
        return _build_one(LIB_OMP, ["-fopenmp"], force)
    return _build_one(LIB, [], force)


def build_all(force: bool = False):
    return build(force), build(force, openmp=True)


if __name__ == "__main__":
    print(build_all(force="--force" in sys.argv))

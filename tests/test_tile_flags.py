"""Host-side check of the 2DSW tile kernel's tables (no GPU needed): the
flag table that tells each row of a tile which phases it takes part in,
and the largest tile heights whose halo still fits the shared arrays.

The tile kernel advances a tile plus a 2T-cell halo T steps per launch;
the region that can still reach the written block shrinks by one row per
phase (three phases per step, Sec. 6.2 of arXiv:1711.04471: the momentum
predictor, continuity, the Shapiro filter).  A row therefore takes part
in phase ph of step t exactly when it is at least 2t + ph rows from both
the top and the bottom edge of the tile.  The table gives that as 9 bits
per distance; this test compiles a host program against the kernel's
header and checks every depth, tile height and row."""
import importlib
import os
import subprocess

import pytest

B = importlib.import_module("paper_1711_04471_gb300.build")   # the build module (the package exports a build function)

PROGRAM = r"""
#include <cstdio>
#include "sw_tile.cuh"
int main()
{
    for (int T = 1; T <= gbsw::SWT_MAX_T; ++T)
        std::printf("%d %d %llu %d %d %d\n", T, gbsw::swt_max_rows(T), (unsigned long long)gbsw::swt_row_bits(T),
                    gbsw::SWT_W, gbsw::SWT_H, gbsw::SWT_NC_MAX);
    return 0;
}
"""


@pytest.fixture(scope="module")
def tables():
    out_dir = os.path.join(B.HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    src = os.path.join(out_dir, "tile_flags_check.cu")
    exe = os.path.join(out_dir, "tile_flags_check")
    with open(src, "w") as f:
        f.write(PROGRAM)
    subprocess.run([B.nvcc(), B.ARCH, "-std=c++17", "-I" + B.CSRC, "-I" + os.path.join(B.ROOT, "include"),
                    src, "-o", exe], check=True, capture_output=True)
    rows = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    return [tuple(int(x) for x in r.split()) for r in rows if r.strip()]


def test_row_flags_follow_the_shrinking_region(tables):
    assert [t[0] for t in tables] == [1, 2, 3]
    for T, max_rows, table, W, H, nc_max in tables:
        assert table < 1 << (9 * (2 * T + 1))
        for th in range(2, max_rows + 1):
            LH = th + 4 * T
            for ly in range(LH):
                d = min(ly, LH - 1 - ly)
                bits = (table >> (9 * min(d, 2 * T))) & 0x1FF
                for t in range(T):
                    for ph in range(3):
                        lo = 2 * t + ph
                        assert bool(bits >> (3 * t + ph) & 1) == (lo <= ly < LH - lo), (T, th, ly, t, ph)
                # bits of steps beyond T are never set
                assert bits >> (3 * T) == 0


def test_largest_tile_heights_fit_the_shared_arrays(tables):
    for T, max_rows, _, W, H, nc_max in tables:
        LW = W + 4 * T
        assert LW * (max_rows + 4 * T) <= nc_max < LW * (max_rows + 1 + 4 * T)
        assert H <= max_rows          # the default tile fits at every depth
    assert [t[1] for t in tables] == [52, 43, 34]

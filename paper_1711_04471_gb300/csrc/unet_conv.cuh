// 3x3x3 convolution of the warm-start U-Net as an implicit GEMM on the
// Blackwell tensor cores (tcgen05, BF16 inputs, FP32 accumulation in TMEM).
//
// Activation layout ("C8-blocked", BF16): element (zn, y, x, c) of a tensor
// with CG = C/8 channel groups sits at (((zn*CG + c/8)*H + y)*W + x)*8 + c%8,
// zn = sample*D + z.  A group of 8 channels of one voxel is 16 bytes, so a
// TMA box {8 ch, box_x, box_y, CG, 1} lands in shared memory as CG slabs of
// 128 voxels x 16 bytes: exactly the no-swizzle K-major canonical layout of
// a 128-row UMMA operand (core matrix = 8 voxels x 8 channels = 128 B, next
// 8 voxels +128 B, next 8 channels +2048 B).  Zero padding at the x/y edges
// comes from the TMA out-of-bounds fill; taps that leave the sample in z are
// skipped (they would read the neighbouring sample).
//
// Weights per tap are packed as [ci/8][co][8] BF16 (the same canonical
// layout with N = Cout rows), copied per tap with one bulk copy.
//
// Small planes (box_x * H < 128, the coarse levels of a network run on a
// coarsened grid) make a tile of box_z consecutive planes of box_y = H rows.
// Each (plane, channel group) is then one TMA box {8, box_x, box_y, 1, 1}
// placed at plane * box_x * box_y * 16 bytes inside its slab, which keeps the
// canonical layout; a plane whose tap leaves its sample, or that lies past
// the last plane, is loaded from z = -1 (all out of bounds: zero fill) and
// its voxels are not stored.
//
// One CTA computes one tile of 128 voxels (box_z x box_y x box_x) and
// all Cout channels: thread 0 of warp 0 issues the loads of tap t into a
// 4-stage ring, thread 0 of warp 1 issues Cin/16 MMAs (M=128, N=Cout, K=16)
// per tap and commits each stage back to the producer, and all four warps
// read the accumulator (warp w owns TMEM lanes 32w..32w+31 = voxels) for
// the epilogue.
//
// Weight gradients (wgrad_tc_kernel) contract over voxels instead:
// dW[tap][co][ci] = sum_v gz[v][co] x[v + off(tap)][ci].  The same
// C8-blocked tiles, read with K = voxels, are MN-major operands (the 8
// channels of a voxel contiguous, consecutive voxels 16 bytes apart): core
// matrix = 8 voxels x 8 channels = 128 B, K step (next 8 voxels) 128 B, MN
// step (next 8 channels) 2048 B.  128 / Cin taps' shifted x tiles, stacked,
// form the 128 rows (tap, ci) of the A operand; the gz tile is B (N = Cout
// rows); every tap's accumulator stays in TMEM while the CTA walks its
// voxel tiles.
#pragma once

#include "common.cuh"
#include "tc.cuh"

namespace gbsw {

struct ConvGeom {
    int NZ, H, W;        // samples*D, rows, columns
    int D;               // depth of one sample
    int box_x, box_y;    // tile = box_z planes x box_y rows x box_x voxels = 128 voxels
    int box_z;           // 1 unless box_x * H < 128
    int tiles_x, tiles_y, tiles_z;
    int out_cg_total, out_cg0;    // output tensor channel groups and offset
    int mask_cg_total, mask_cg0;  // mask tensor (EPI_MASK)
};

// Arguments of one weight-gradient launch (dw accumulates with atomics:
// zero it first).  xmap: the layer input (Cin channels), gmap: the
// gradient of the layer output before the bias (Cout channels), both
// C8-blocked with the forward conv's boxes; only input channels
// ci < cin_store are written, at dw[(tap * Cout + co) * cin_store + ci].
struct WgradCall {
    CUtensorMap xmap, gmap;
    ConvGeom geom;
    float *dw;
    int cin_store;
    int *status;
};

enum ConvEpilogue : int {
    EPI_BIAS_RELU = 0,  // y = max(acc + bias, 0)
    EPI_RAW = 1,        // y = acc
    EPI_MASK = 2        // y = acc * [mask > 0]  (backward through a ReLU)
};

}  // namespace gbsw

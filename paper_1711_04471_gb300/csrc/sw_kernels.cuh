// Device kernels of the 2-D shallow-water step (Sec. 6.2 of arXiv:1711.04471).
//
// Device layout: every field is an ny x pitch FP32 array (pitch = nx rounded
// up to 32 floats, rows 128-byte aligned), 0-based cell (i, j) at
// j*pitch + i.  eta and H live at cell centres, u[j][i] on the east face
// and v[j][i] on the north face of cell (i, j).  The west and south walls
// are not stored (they are identically 0); the east column i = nx-1 of u
// and the north row j = ny-1 of v are the other two walls and stay 0.
// Cells outside the domain read as H = eta = 0, i.e. dry.  The fused
// time-step kernel is in sw_stream.cuh.
#pragma once

#include "common.cuh"

namespace gbsw {

struct SWDev {
    int nx, ny, pitch;
    float gdt_dx, gdt_dy;  // g*dt/dx, g*dt/dy
    float dt_dx, dt_dy;    // dt/dx, dt/dy
    float q;               // eps/4, the Shapiro neighbour weight
    float hmin;            // wet threshold
};

constexpr int SW_MAX_BLOCKING = 6;   // deepest temporal blocking compiled
constexpr int SW_VOL_BLOCKS = 1024;  // fixed, so the FP64 sum order is fixed
constexpr int SW_VOL_THREADS = 256;
constexpr int SW_NOALLOC_MAX_SIDE = 1 << 20;  // largest nx, ny accepted by sw_volume_noalloc

// Out-of-range index count of the bounds-checked debug build (one per
// translation unit that includes this header).
static __device__ unsigned g_sw_bounds;

// Wet/dry face rule: keep the predicted velocity if both cells are wet, or
// if it flows out of a wet cell; otherwise the face is closed.
__device__ __forceinline__ float sw_face_mask(float vel, bool wet_behind, bool wet_ahead)
{
    const bool keep = (wet_behind && wet_ahead) || (wet_behind && vel > 0.0f) || (wet_ahead && vel < 0.0f);
    return keep ? vel : 0.0f;
}

// The step's arithmetic is written with explicit round-to-nearest
// intrinsics (no compiler-chosen multiply-add contraction), so the result
// of a cell does not depend on the fusion depth or the tiling.
__device__ __forceinline__ float sw_upwind(float vel, float h_behind, float h_ahead)
{
    return __fmaf_rn(fmaxf(vel, 0.0f), h_behind, __fmul_rn(fminf(vel, 0.0f), h_ahead));
}

// u - c (e_ahead - e_behind): the momentum predictor of one face.
__device__ __forceinline__ float sw_predict(float vel, float c, float e_ahead, float e_behind)
{
    return __fmaf_rn(-c, __fsub_rn(e_ahead, e_behind), vel);
}

}  // namespace gbsw

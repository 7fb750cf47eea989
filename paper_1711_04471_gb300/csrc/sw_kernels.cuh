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

// Wet/dry face rule: keep the predicted velocity if both cells are wet, or
// if it flows out of a wet cell; otherwise the face is closed.
__device__ __forceinline__ float sw_face_mask(float vel, bool wet_behind, bool wet_ahead)
{
    const bool keep = (wet_behind && wet_ahead) || (wet_behind && vel > 0.0f) || (wet_ahead && vel < 0.0f);
    return keep ? vel : 0.0f;
}

__device__ __forceinline__ float sw_upwind(float vel, float h_behind, float h_ahead)
{
    return fmaxf(vel, 0.0f) * h_behind + fminf(vel, 0.0f) * h_ahead;
}

// FP64 volume partial sums over rows blockIdx.x, blockIdx.x + gridDim.x, ...
// partials[3*b + {0,1,2}] = sum h, sum of h over wet cells, count of
// non-finite eta.  The order of every sum depends only on (nx, ny).
__global__ void __launch_bounds__(SW_VOL_THREADS)
sw_volume_partial_kernel(SWDev p, const float *__restrict__ H, const float *__restrict__ eta,
                         double *__restrict__ partials)
{
    __shared__ double red[SW_VOL_THREADS / 32];
    double s = 0.0, sw = 0.0, bad = 0.0;
    for (int j = blockIdx.x; j < p.ny; j += gridDim.x) {
        const size_t row = (size_t)j * p.pitch;
        for (int i = threadIdx.x; i < p.nx; i += blockDim.x) {
            const float e = eta[row + i], hh = H[row + i];
            if (!isfinite(e)) bad += 1.0;
            const double h = (double)hh + (double)e;
            s += h;
            if (hh + e > p.hmin) sw += h;
        }
    }
    s = block_sum_f64<SW_VOL_THREADS / 32>(s, red);
    sw = block_sum_f64<SW_VOL_THREADS / 32>(sw, red);
    bad = block_sum_f64<SW_VOL_THREADS / 32>(bad, red);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = s;
        partials[3 * blockIdx.x + 1] = sw;
        partials[3 * blockIdx.x + 2] = bad;
    }
}

// Second pass: one block folds the partials in a fixed order and scales.
__global__ void __launch_bounds__(SW_VOL_THREADS)
sw_volume_final_kernel(const double *__restrict__ partials, int nblocks, double area, double *__restrict__ out)
{
    __shared__ double red[SW_VOL_THREADS / 32];
    double s = 0.0, sw = 0.0, bad = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        s += partials[3 * b + 0];
        sw += partials[3 * b + 1];
        bad += partials[3 * b + 2];
    }
    s = block_sum_f64<SW_VOL_THREADS / 32>(s, red);
    sw = block_sum_f64<SW_VOL_THREADS / 32>(sw, red);
    bad = block_sum_f64<SW_VOL_THREADS / 32>(bad, red);
    if (threadIdx.x == 0) {
        out[0] = s * area;
        out[1] = sw * area;
        out[2] = bad;
    }
}

// Wet mask as bytes (packed nx per row) for host read-back.
__global__ void sw_wet_mask_kernel(SWDev p, const float *__restrict__ H, const float *__restrict__ eta,
                                   uint8_t *__restrict__ wet)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= p.nx || j >= p.ny) return;
    const size_t g = (size_t)j * p.pitch + i;
    wet[(size_t)j * p.nx + i] = H[g] + eta[g] > p.hmin;
}

}  // namespace gbsw

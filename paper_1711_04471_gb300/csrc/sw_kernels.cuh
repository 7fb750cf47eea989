// Device kernels of the 2-D shallow-water step (Sec. 6.2 of arXiv:1711.04471).
//
// Device layout: every field is an ny x pitch FP32 array (pitch = nx rounded
// up to 32 floats, rows 128-byte aligned), 0-based cell (i, j) at
// j*pitch + i.  eta and H live at cell centres, u[j][i] on the east face
// and v[j][i] on the north face of cell (i, j).  The west and south walls
// are not stored (they are identically 0); the east column i = nx-1 of u
// and the north row j = ny-1 of v are the other two walls and stay 0.
// Cells outside the domain read as H = eta = 0, i.e. dry.
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

constexpr int SW_BLOCK_Y = 8;        // blocks are 32 x 8 threads
constexpr int SW_MAX_BLOCKING = 4;   // deepest temporal blocking compiled
constexpr int SW_VOL_BLOCKS = 1024;  // fixed, so the FP64 sum order is fixed
constexpr int SW_VOL_THREADS = 256;
constexpr int SW_NOALLOC_MAX_SIDE = 1 << 20;  // largest nx, ny accepted by sw_volume_noalloc

template <int T, int TX, int TY>
struct SWTile {
    static constexpr int R = 2 * T;          // halo: 2 cells per fused step
    static constexpr int RX = TX + 2 * R;
    static constexpr int RY = TY + 2 * R;
    static constexpr int N = RX * RY;
    // eta, H, u, v, eta* (FP32) + wet (byte) per region cell
    static constexpr size_t smem_bytes = (size_t)N * (5 * sizeof(float) + 1);
};

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

// T fused time steps over a TX x TY tile.  Launch: grid (ceil(nx/TX),
// ceil(ny/TY)), block (32, SW_BLOCK_Y), dynamic smem SWTile::smem_bytes.
template <int T, int TX, int TY>
__global__ void __launch_bounds__(32 * SW_BLOCK_Y)
sw_fused_kernel(SWDev p, const float *__restrict__ H, const float *__restrict__ eta_in,
                const float *__restrict__ u_in, const float *__restrict__ v_in, float *__restrict__ eta_out,
                float *__restrict__ u_out, float *__restrict__ v_out)
{
    using Tile = SWTile<T, TX, TY>;
    constexpr int R = Tile::R, RX = Tile::RX, RY = Tile::RY, N = Tile::N;
    extern __shared__ float smem[];
    float *s_eta = smem;
    float *s_H = s_eta + N;
    float *s_u = s_H + N;
    float *s_v = s_u + N;
    float *s_es = s_v + N;
    uint8_t *s_wet = reinterpret_cast<uint8_t *>(s_es + N);

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int i0 = blockIdx.x * TX - R;  // global index of region column 0
    const int j0 = blockIdx.y * TY - R;
    const int nx = p.nx, ny = p.ny;

    for (int y = ty; y < RY; y += SW_BLOCK_Y) {
        const int gj = j0 + y;
        const bool row_in = gj >= 0 && gj < ny;
        const size_t grow = (size_t)(row_in ? gj : 0) * p.pitch;
        for (int x = tx; x < RX; x += 32) {
            const int gi = i0 + x;
            const bool in = row_in && gi >= 0 && gi < nx;
            const int s = y * RX + x;
            s_eta[s] = in ? __ldg(eta_in + grow + gi) : 0.0f;
            s_H[s] = in ? __ldg(H + grow + gi) : 0.0f;
            s_u[s] = in ? __ldg(u_in + grow + gi) : 0.0f;
            s_v[s] = in ? __ldg(v_in + grow + gi) : 0.0f;
        }
    }
    __syncthreads();

    const float hmin = p.hmin;
#pragma unroll 1
    for (int st = 0; st < T; ++st) {
        const int lo = 2 * st;
        // (dyn, momentum) u' on east faces of cells x in [lo, RX-lo-1), v' on
        // north faces of cells y in [lo, RY-lo-1); updated in place.
        for (int y = lo + ty; y < RY - lo; y += SW_BLOCK_Y) {
            const int gj = j0 + y;
            for (int x = lo + tx; x < RX - lo; x += 32) {
                const int s = y * RX + x;
                const int gi = i0 + x;
                const float ec = s_eta[s];
                const bool wc = s_H[s] + ec > hmin;
                if (x < RX - lo - 1) {
                    float un = 0.0f;
                    if (gi >= 0 && gi < nx - 1) {
                        const float ee = s_eta[s + 1];
                        const bool we = s_H[s + 1] + ee > hmin;
                        un = sw_face_mask(s_u[s] - p.gdt_dx * (ee - ec), wc, we);
                    }
                    s_u[s] = un;
                }
                if (y < RY - lo - 1) {
                    float vn = 0.0f;
                    if (gj >= 0 && gj < ny - 1) {
                        const float en = s_eta[s + RX];
                        const bool wn = s_H[s + RX] + en > hmin;
                        vn = sw_face_mask(s_v[s] - p.gdt_dy * (en - ec), wc, wn);
                    }
                    s_v[s] = vn;
                }
            }
        }
        __syncthreads();
        // (dyn, continuity) eta* on cells [lo+1, R?-lo-1); also the wet mask
        // of the start of the step for the filter.
        for (int y = lo + 1 + ty; y < RY - lo - 1; y += SW_BLOCK_Y) {
            for (int x = lo + 1 + tx; x < RX - lo - 1; x += 32) {
                const int s = y * RX + x;
                const float hc = s_H[s] + s_eta[s];
                const float he = s_H[s + 1] + s_eta[s + 1];
                const float hw = s_H[s - 1] + s_eta[s - 1];
                const float hn = s_H[s + RX] + s_eta[s + RX];
                const float hs = s_H[s - RX] + s_eta[s - RX];
                const float fe = sw_upwind(s_u[s], hc, he);
                const float fw = sw_upwind(s_u[s - 1], hw, hc);
                const float gn = sw_upwind(s_v[s], hc, hn);
                const float gs = sw_upwind(s_v[s - RX], hs, hc);
                s_es[s] = s_eta[s] - (p.dt_dx * (fe - fw) + p.dt_dy * (gn - gs));
                s_wet[s] = hc > hmin;
            }
        }
        __syncthreads();
        // (shapiro) eta+ on cells [lo+2, R?-lo-2), then eta <- eta+.
        for (int y = lo + 2 + ty; y < RY - lo - 2; y += SW_BLOCK_Y) {
            for (int x = lo + 2 + tx; x < RX - lo - 2; x += 32) {
                const int s = y * RX + x;
                const float es = s_es[s];
                float out = es;
                if (s_wet[s]) {
                    const float we = s_wet[s + 1], ww = s_wet[s - 1], wn = s_wet[s + RX], ws = s_wet[s - RX];
                    const float cnt = (we + ww) + (wn + ws);
                    const float sum = (we * s_es[s + 1] + ww * s_es[s - 1]) + (wn * s_es[s + RX] + ws * s_es[s - RX]);
                    out = (1.0f - p.q * cnt) * es + p.q * sum;
                }
                s_eta[s] = out;
            }
        }
        __syncthreads();
    }

    for (int y = R + ty; y < R + TY; y += SW_BLOCK_Y) {
        const int gj = j0 + y;
        if (gj >= ny) break;
        const size_t grow = (size_t)gj * p.pitch;
        for (int x = R + tx; x < R + TX; x += 32) {
            const int gi = i0 + x;
            if (gi >= nx) break;
            const int s = y * RX + x;
            eta_out[grow + gi] = s_eta[s];
            u_out[grow + gi] = s_u[s];
            v_out[grow + gi] = s_v[s];
        }
    }
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

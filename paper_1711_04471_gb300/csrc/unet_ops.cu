// U-Net glue kernels: the first (2-channel) convolution on CUDA cores,
// pooling / upsampling in the C8-blocked layout, the 1x1 head with the MSE
// loss, weight gradients and Adam.
#include <algorithm>

#include "unet_ops.cuh"

namespace gbsw {

__device__ __forceinline__ size_t bidx(int zn, int cg_total, int cg, int H, int W, int y, int x)
{
    return ((((size_t)zn * cg_total + cg) * H + y) * W + x) * 8;
}

// ---------------------------------------------------------------- layer l1a
// y = relu(conv(x) + b) with x dense FP32 (zn, y, x, 2), 16 outputs into a
// C8-blocked tensor.  One thread per voxel; weights in shared memory.
__global__ void conv_in2_kernel(const float *__restrict__ x, const float *__restrict__ w, const float *__restrict__ b,
                                int NZ, int D, int H, int W, __nv_bfloat16 *__restrict__ y, int cg_total, int cg0)
{
    __shared__ float sw[27 * 16 * 2];
    __shared__ float sb[16];
    for (int q = threadIdx.x; q < 27 * 32; q += blockDim.x) sw[q] = w[q];
    if (threadIdx.x < 16) sb[threadIdx.x] = b[threadIdx.x];
    __syncthreads();
    const long long n = (long long)NZ * H * W;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int xx = (int)(v % W);
    const int yy = (int)((v / W) % H);
    const int zn = (int)(v / ((long long)W * H));
    const int z = zn % D;
    float acc[16];
#pragma unroll
    for (int co = 0; co < 16; ++co) acc[co] = sb[co];
    for (int tap = 0; tap < 27; ++tap) {
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        if (z + dz < 0 || z + dz >= D || yy + dy < 0 || yy + dy >= H || xx + dx < 0 || xx + dx >= W) continue;
        const float2 in = *reinterpret_cast<const float2 *>(x + ((((size_t)(zn + dz) * H) + yy + dy) * W + xx + dx) * 2);
#pragma unroll
        for (int co = 0; co < 16; ++co) acc[co] += sw[(tap * 16 + co) * 2] * in.x + sw[(tap * 16 + co) * 2 + 1] * in.y;
    }
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        uint4 pk;
        __nv_bfloat162 *p2 = reinterpret_cast<__nv_bfloat162 *>(&pk);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            p2[q] = __floats2bfloat162_rn(fmaxf(acc[g * 8 + 2 * q], 0.0f), fmaxf(acc[g * 8 + 2 * q + 1], 0.0f));
        *reinterpret_cast<uint4 *>(y + bidx(zn, cg_total, cg0 + g, H, W, yy, xx)) = pk;
    }
}

// dW of l1a: dw[tap][co][ci] += sum_v g[v, co] x[v + off(tap), ci], db[co] += sum_v g[v, co].
// grid (27, chunks), block 256; g is C8-blocked (16 ch), x dense FP32 (2 ch).
__global__ void wgrad_in2_kernel(const float *__restrict__ x, const __nv_bfloat16 *__restrict__ g, int g_cg_total,
                                 int g_cg0, int NZ, int D, int H, int W, float *__restrict__ dw, float *__restrict__ db)
{
    const int tap = blockIdx.x;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    float acc[32];
    float accb[16];
#pragma unroll
    for (int q = 0; q < 32; ++q) acc[q] = 0.0f;
#pragma unroll
    for (int q = 0; q < 16; ++q) accb[q] = 0.0f;
    const long long n = (long long)NZ * H * W;
    for (long long v = (long long)blockIdx.y * blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.y * blockDim.x) {
        const int xx = (int)(v % W);
        const int yy = (int)((v / W) % H);
        const int zn = (int)(v / ((long long)W * H));
        const int z = zn % D;
        float gv[16];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const uint4 pk = *reinterpret_cast<const uint4 *>(g + bidx(zn, g_cg_total, g_cg0 + c, H, W, yy, xx));
            const __nv_bfloat16 *pb = reinterpret_cast<const __nv_bfloat16 *>(&pk);
#pragma unroll
            for (int q = 0; q < 8; ++q) gv[c * 8 + q] = __bfloat162float(pb[q]);
        }
        if (tap == 13)
#pragma unroll
            for (int q = 0; q < 16; ++q) accb[q] += gv[q];
        if (z + dz < 0 || z + dz >= D || yy + dy < 0 || yy + dy >= H || xx + dx < 0 || xx + dx >= W) continue;
        const float2 in = *reinterpret_cast<const float2 *>(x + ((((size_t)(zn + dz) * H) + yy + dy) * W + xx + dx) * 2);
#pragma unroll
        for (int co = 0; co < 16; ++co) {
            acc[co * 2] += gv[co] * in.x;
            acc[co * 2 + 1] += gv[co] * in.y;
        }
    }
    __shared__ float red[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 32; ++q) {
        float s = acc[q];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp][q] = s;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        float s = 0.0f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k][threadIdx.x];
        atomicAdd(&dw[tap * 32 + threadIdx.x], s);
    }
    if (tap == 13) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            float s = accb[q];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (lane == 0) red[warp][q] = s;
        }
        __syncthreads();
        if (threadIdx.x < 16) {
            float s = 0.0f;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k][threadIdx.x];
            atomicAdd(&db[threadIdx.x], s);
        }
    }
}

// ------------------------------------------------------------ weight grads
// dw[tap][co][ci] += sum_v g[v, co] x[v + off(tap), ci] for one tap per
// grid-x index, over the 128-voxel tiles of chunk blockIdx.y; db from the
// centre tap.  x and g are C8-blocked.  Shared memory holds one tile of
// g (FP32) and the tap-shifted tile of x (FP32, zero outside the sample).
template <int CIN, int COUT>
__global__ void __launch_bounds__(256)
wgrad_kernel(const __nv_bfloat16 *__restrict__ x, int x_cg_total, int x_cg0, const __nv_bfloat16 *__restrict__ g,
             int g_cg_total, int g_cg0, ConvGeom geo, int tiles_per_cta, float *__restrict__ dw, float *__restrict__ db)
{
    constexpr int OUT = CIN * COUT;
    constexpr int PER = (OUT + 255) / 256;  // outputs per thread
    __shared__ float sg[64][COUT + 1];  // half a tile at a time (fits the 48 KB static limit)
    __shared__ float sx[64][CIN + 1];
    const int tap = blockIdx.x;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int ntiles = geo.tiles_z * geo.tiles_y * geo.tiles_x;
    const int plane = geo.box_x * geo.box_y;  // voxels of one plane of a tile
    float acc[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) acc[q] = 0.0f;
    float accb = 0.0f;
    for (int t = blockIdx.y * tiles_per_cta; t < min(ntiles, (blockIdx.y + 1) * tiles_per_cta); ++t) {
        int tt = t;
        const int tx = tt % geo.tiles_x;
        tt /= geo.tiles_x;
        const int ty = tt % geo.tiles_y;
        const int z0 = (tt / geo.tiles_y) * geo.box_z;
        const int x0 = tx * geo.box_x, y0 = ty * geo.box_y;
        for (int half = 0; half < 2; ++half) {
            __syncthreads();
            // stage 64 voxels: one thread per (voxel, channel group)
            for (int q = threadIdx.x; q < 64 * (COUT / 8); q += 256) {
                const int mm = q % 64, cb = q / 64, m = half * 64 + mm;
                const int zn = z0 + m / plane, r = m % plane;
                const int yy = y0 + r / geo.box_x, xx = x0 + r % geo.box_x;
                uint4 pk = make_uint4(0, 0, 0, 0);  // voxels past the last plane contribute nothing
                if (zn < geo.NZ)
                    pk = *reinterpret_cast<const uint4 *>(g + bidx(zn, g_cg_total, g_cg0 + cb, geo.H, geo.W, yy, xx));
                const __nv_bfloat16 *pb = reinterpret_cast<const __nv_bfloat16 *>(&pk);
#pragma unroll
                for (int k = 0; k < 8; ++k) sg[mm][cb * 8 + k] = __bfloat162float(pb[k]);
            }
            for (int q = threadIdx.x; q < 64 * (CIN / 8); q += 256) {
                const int mm = q % 64, cb = q / 64, m = half * 64 + mm;
                const int zn = z0 + m / plane, r = m % plane, z = zn % geo.D;
                const int yy = y0 + r / geo.box_x + dy, xx = x0 + r % geo.box_x + dx;
                const bool in = zn < geo.NZ && z + dz >= 0 && z + dz < geo.D && yy >= 0 && yy < geo.H && xx >= 0 &&
                                xx < geo.W;
                uint4 pk = make_uint4(0, 0, 0, 0);
                if (in)
                    pk = *reinterpret_cast<const uint4 *>(
                        x + bidx(zn + dz, x_cg_total, x_cg0 + cb, geo.H, geo.W, yy, xx));
                const __nv_bfloat16 *pb = reinterpret_cast<const __nv_bfloat16 *>(&pk);
#pragma unroll
                for (int k = 0; k < 8; ++k) sx[mm][cb * 8 + k] = __bfloat162float(pb[k]);
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int o = threadIdx.x + q * 256;
                if (o < OUT) {
                    const int co = o / CIN, ci = o % CIN;
                    float sacc = 0.0f;
#pragma unroll 8
                    for (int m = 0; m < 64; ++m) sacc += sg[m][co] * sx[m][ci];
                    acc[q] += sacc;
                }
            }
            if (tap == 13 && threadIdx.x < COUT)
                for (int m = 0; m < 64; ++m) accb += sg[m][threadIdx.x];
        }
    }
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int o = threadIdx.x + q * 256;
        if (o < OUT) atomicAdd(&dw[(size_t)tap * OUT + o], acc[q]);
    }
    if (tap == 13 && threadIdx.x < COUT) atomicAdd(&db[threadIdx.x], accb);
}

// ------------------------------------------------------- pool / upsample
// y = 2x2x2 average of x (level sizes: x is (NZ, H, W), y is (NZ/2, H/2, W/2)).
__global__ void pool_kernel(const __nv_bfloat16 *__restrict__ x, int x_cg_total, int x_cg0, int NZ, int H, int W,
                            int C, __nv_bfloat16 *__restrict__ y, int y_cg_total, int y_cg0)
{
    const int h = H / 2, w = W / 2;
    const long long n = (long long)(NZ / 2) * h * w * (C / 8);
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int xx = (int)(q % w);
    long long r = q / w;
    const int yy = (int)(r % h);
    r /= h;
    const int cb = (int)(r % (C / 8));
    const int zn = (int)(r / (C / 8));
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 8; ++k) {
        const uint4 pk = *reinterpret_cast<const uint4 *>(
            x + bidx(2 * zn + (k >> 2), x_cg_total, x_cg0 + cb, H, W, 2 * yy + ((k >> 1) & 1), 2 * xx + (k & 1)));
        const __nv_bfloat16 *pb = reinterpret_cast<const __nv_bfloat16 *>(&pk);
#pragma unroll
        for (int c = 0; c < 8; ++c) s[c] += __bfloat162float(pb[c]);
    }
    uint4 out;
    __nv_bfloat162 *p2 = reinterpret_cast<__nv_bfloat162 *>(&out);
#pragma unroll
    for (int c = 0; c < 4; ++c) p2[c] = __floats2bfloat162_rn(0.125f * s[2 * c], 0.125f * s[2 * c + 1]);
    *reinterpret_cast<uint4 *>(y + bidx(zn, y_cg_total, y_cg0 + cb, h, w, yy, xx)) = out;
}

// y (2NZ, 2H, 2W) = nearest upsampling of x (NZ, H, W).
__global__ void upsample_kernel(const __nv_bfloat16 *__restrict__ x, int x_cg_total, int x_cg0, int NZ, int H, int W,
                                int C, __nv_bfloat16 *__restrict__ y, int y_cg_total, int y_cg0)
{
    const int H2 = 2 * H, W2 = 2 * W;
    const long long n = (long long)(2 * NZ) * H2 * W2 * (C / 8);
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int xx = (int)(q % W2);
    long long r = q / W2;
    const int yy = (int)(r % H2);
    r /= H2;
    const int cb = (int)(r % (C / 8));
    const int zn = (int)(r / (C / 8));
    *reinterpret_cast<uint4 *>(y + bidx(zn, y_cg_total, y_cg0 + cb, H2, W2, yy, xx)) =
        *reinterpret_cast<const uint4 *>(x + bidx(zn / 2, x_cg_total, x_cg0 + cb, H, W, yy / 2, xx / 2));
}

// Adjoint of upsample: y (NZ, H, W) = sum of the 8 children in x (2NZ, 2H, 2W).
__global__ void upsample_bwd_kernel(const __nv_bfloat16 *__restrict__ x, int x_cg_total, int x_cg0, int NZ, int H, int W,
                                    int C, __nv_bfloat16 *__restrict__ y, int y_cg_total, int y_cg0)
{
    const long long n = (long long)NZ * H * W * (C / 8);
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int xx = (int)(q % W);
    long long r = q / W;
    const int yy = (int)(r % H);
    r /= H;
    const int cb = (int)(r % (C / 8));
    const int zn = (int)(r / (C / 8));
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 8; ++k) {
        const uint4 pk = *reinterpret_cast<const uint4 *>(
            x + bidx(2 * zn + (k >> 2), x_cg_total, x_cg0 + cb, 2 * H, 2 * W, 2 * yy + ((k >> 1) & 1), 2 * xx + (k & 1)));
        const __nv_bfloat16 *pb = reinterpret_cast<const __nv_bfloat16 *>(&pk);
#pragma unroll
        for (int c = 0; c < 8; ++c) s[c] += __bfloat162float(pb[c]);
    }
    uint4 out;
    __nv_bfloat162 *p2 = reinterpret_cast<__nv_bfloat162 *>(&out);
#pragma unroll
    for (int c = 0; c < 4; ++c) p2[c] = __floats2bfloat162_rn(s[2 * c], s[2 * c + 1]);
    *reinterpret_cast<uint4 *>(y + bidx(zn, y_cg_total, y_cg0 + cb, H, W, yy, xx)) = out;
}

// Gradient of a ReLU output that feeds both a concatenation and a pool:
// out (NZ, H, W) = (from_cat + pool_bwd(from_pool)) * [act > 0],
// from_pool at (NZ/2, H/2, W/2).
__global__ void pool_bwd_add_mask_kernel(const __nv_bfloat16 *__restrict__ from_cat, int c_cg_total, int c_cg0,
                                         const __nv_bfloat16 *__restrict__ from_pool, int p_cg_total, int p_cg0,
                                         const __nv_bfloat16 *__restrict__ act, int a_cg_total, int a_cg0, int NZ, int H,
                                         int W, int C, __nv_bfloat16 *__restrict__ out, int o_cg_total, int o_cg0)
{
    const long long n = (long long)NZ * H * W * (C / 8);
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int xx = (int)(q % W);
    long long r = q / W;
    const int yy = (int)(r % H);
    r /= H;
    const int cb = (int)(r % (C / 8));
    const int zn = (int)(r / (C / 8));
    const uint4 a = *reinterpret_cast<const uint4 *>(from_cat + bidx(zn, c_cg_total, c_cg0 + cb, H, W, yy, xx));
    const uint4 b = *reinterpret_cast<const uint4 *>(
        from_pool + bidx(zn / 2, p_cg_total, p_cg0 + cb, H / 2, W / 2, yy / 2, xx / 2));
    const uint4 m = *reinterpret_cast<const uint4 *>(act + bidx(zn, a_cg_total, a_cg0 + cb, H, W, yy, xx));
    const __nv_bfloat16 *pa = reinterpret_cast<const __nv_bfloat16 *>(&a);
    const __nv_bfloat16 *pb = reinterpret_cast<const __nv_bfloat16 *>(&b);
    const __nv_bfloat16 *pm = reinterpret_cast<const __nv_bfloat16 *>(&m);
    uint4 o;
    __nv_bfloat16 *po = reinterpret_cast<__nv_bfloat16 *>(&o);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const float v = __bfloat162float(pa[c]) + 0.125f * __bfloat162float(pb[c]);
        po[c] = __float2bfloat16_rn(__bfloat162float(pm[c]) > 0.0f ? v : 0.0f);
    }
    *reinterpret_cast<uint4 *>(out + bidx(zn, o_cg_total, o_cg0 + cb, H, W, yy, xx)) = o;
}

// ------------------------------------------------------------------ head
// out[v] = sum_c d1[v, c] hw[c] + hb (16 -> 1, no activation).
__global__ void head_fwd_kernel(const __nv_bfloat16 *__restrict__ d1, int cg_total, int cg0, long long nvox, int H,
                                int W, const float *__restrict__ hw, const float *__restrict__ hb, float *__restrict__ out)
{
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const int xx = (int)(v % W);
    const int yy = (int)((v / W) % H);
    const int zn = (int)(v / ((long long)W * H));
    float s = hb[0];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const uint4 pk = *reinterpret_cast<const uint4 *>(d1 + bidx(zn, cg_total, cg0 + c, H, W, yy, xx));
        const __nv_bfloat16 *pb = reinterpret_cast<const __nv_bfloat16 *>(&pk);
#pragma unroll
        for (int q = 0; q < 8; ++q) s += __bfloat162float(pb[q]) * hw[c * 8 + q];
    }
    out[v] = s;
}

// MSE loss and the head's backward pass:
//   dout = 2 (out - t) / nvox;  loss += sum (out - t)^2 / nvox (FP64)
//   g_hw[c] += sum dout d1[c];  g_hb += sum dout
//   g_d1[v, c] = dout hw[c] [d1[v, c] > 0]   (C8-blocked, the gz of l1c)
__global__ void __launch_bounds__(256)
head_bwd_kernel(const __nv_bfloat16 *__restrict__ d1, int cg_total, int cg0, long long nvox, int H, int W,
                const float *__restrict__ out, const float *__restrict__ target, const float *__restrict__ hw,
                float *__restrict__ g_hw, float *__restrict__ g_hb, __nv_bfloat16 *__restrict__ g_d1, double *loss)
{
    __shared__ float red[8][17];
    __shared__ double redl[8];
    float acc[17];
#pragma unroll
    for (int q = 0; q < 17; ++q) acc[q] = 0.0f;
    double l = 0.0;
    const float inv = 1.0f / (float)nvox;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        const int xx = (int)(v % W);
        const int yy = (int)((v / W) % H);
        const int zn = (int)(v / ((long long)W * H));
        const float diff = out[v] - target[v];
        l += (double)diff * (double)diff;
        const float dout = 2.0f * diff * inv;
        acc[16] += dout;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const size_t a = bidx(zn, cg_total, cg0 + c, H, W, yy, xx);
            const uint4 pk = *reinterpret_cast<const uint4 *>(d1 + a);
            const __nv_bfloat16 *pb = reinterpret_cast<const __nv_bfloat16 *>(&pk);
            uint4 go;
            __nv_bfloat16 *pg = reinterpret_cast<__nv_bfloat16 *>(&go);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float dv = __bfloat162float(pb[q]);
                acc[c * 8 + q] += dout * dv;
                pg[q] = __float2bfloat16_rn(dv > 0.0f ? dout * hw[c * 8 + q] : 0.0f);
            }
            *reinterpret_cast<uint4 *>(g_d1 + a) = go;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 17; ++q) {
        float s = acc[q];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) red[warp][q] = s;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if (lane == 0) redl[warp] = l;
    __syncthreads();
    if (threadIdx.x < 17) {
        float s = 0.0f;
        for (int k = 0; k < 8; ++k) s += red[k][threadIdx.x];
        atomicAdd(threadIdx.x < 16 ? &g_hw[threadIdx.x] : g_hb, s);
    }
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += redl[k];
        atomicAdd(loss, s / (double)nvox);
    }
}

// ------------------------------------------------------------------ Adam
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.0f - b1) * gq;
    const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

}  // namespace gbsw

// ----------------------------------------------------------------- launches
namespace gbsw {

namespace {
inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }
}  // namespace

gbsw_status launch_conv_in2(const float *x, const float *w, const float *b, const ConvGeom &g, bf16 *y, int cg_total,
                            int cg0, cudaStream_t s)
{
    const long long n = (long long)g.NZ * g.H * g.W;
    conv_in2_kernel<<<nblk(n, 128), 128, 0, s>>>(x, w, b, g.NZ, g.D, g.H, g.W, y, cg_total, cg0);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status launch_wgrad_in2(const float *x, const bf16 *g, int g_cg_total, int g_cg0, const ConvGeom &geo, float *dw,
                             float *db, cudaStream_t s)
{
    const long long n = (long long)geo.NZ * geo.H * geo.W;
    const int chunks = (int)std::min<long long>(64, std::max<long long>(1, n / (256 * 16)));
    wgrad_in2_kernel<<<dim3(27, chunks), 256, 0, s>>>(x, g, g_cg_total, g_cg0, geo.NZ, geo.D, geo.H, geo.W, dw, db);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status launch_wgrad(int cin, int cout, const bf16 *x, int x_cg_total, int x_cg0, const bf16 *g, int g_cg_total,
                         int g_cg0, const ConvGeom &geo, float *dw, float *db, cudaStream_t s)
{
    const int ntiles = geo.tiles_z * geo.tiles_y * geo.tiles_x;
    const int chunks = std::max(1, std::min(ntiles, 4 * sm_count() / 27 + 1));
    const int per = ceil_div(ntiles, chunks);
    const dim3 grid(27, ceil_div(ntiles, per));
#define WG_CASE(A, B)                                                                                               \
    if (cin == A && cout == B) {                                                                                    \
        wgrad_kernel<A, B><<<grid, 256, 0, s>>>(x, x_cg_total, x_cg0, g, g_cg_total, g_cg0, geo, per, dw, db);      \
        GBSW_LAUNCH_CHECK();                                                                                        \
        return GBSW_OK;                                                                                             \
    }
    WG_CASE(16, 16)
    WG_CASE(16, 32)
    WG_CASE(32, 32)
    WG_CASE(32, 64)
    WG_CASE(64, 32)
    WG_CASE(64, 16)
    WG_CASE(32, 16)
#undef WG_CASE
    return GBSW_ERR_ARG;
}

gbsw_status launch_pool(const bf16 *x, int x_cg_total, int x_cg0, int NZ, int H, int W, int C, bf16 *y, int y_cg_total,
                        int y_cg0, cudaStream_t s)
{
    const long long n = (long long)(NZ / 2) * (H / 2) * (W / 2) * (C / 8);
    pool_kernel<<<nblk(n, 256), 256, 0, s>>>(x, x_cg_total, x_cg0, NZ, H, W, C, y, y_cg_total, y_cg0);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status launch_upsample(const bf16 *x, int x_cg_total, int x_cg0, int NZ, int H, int W, int C, bf16 *y,
                            int y_cg_total, int y_cg0, cudaStream_t s)
{
    const long long n = (long long)(2 * NZ) * (2 * H) * (2 * W) * (C / 8);
    upsample_kernel<<<nblk(n, 256), 256, 0, s>>>(x, x_cg_total, x_cg0, NZ, H, W, C, y, y_cg_total, y_cg0);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status launch_upsample_bwd(const bf16 *x, int x_cg_total, int x_cg0, int NZ, int H, int W, int C, bf16 *y,
                                int y_cg_total, int y_cg0, cudaStream_t s)
{
    const long long n = (long long)NZ * H * W * (C / 8);
    upsample_bwd_kernel<<<nblk(n, 256), 256, 0, s>>>(x, x_cg_total, x_cg0, NZ, H, W, C, y, y_cg_total, y_cg0);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status launch_pool_bwd_add_mask(const bf16 *from_cat, int c_cg_total, int c_cg0, const bf16 *from_pool,
                                     int p_cg_total, int p_cg0, const bf16 *act, int a_cg_total, int a_cg0, int NZ,
                                     int H, int W, int C, bf16 *out, int o_cg_total, int o_cg0, cudaStream_t s)
{
    const long long n = (long long)NZ * H * W * (C / 8);
    pool_bwd_add_mask_kernel<<<nblk(n, 256), 256, 0, s>>>(from_cat, c_cg_total, c_cg0, from_pool, p_cg_total, p_cg0,
                                                          act, a_cg_total, a_cg0, NZ, H, W, C, out, o_cg_total, o_cg0);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status launch_head_fwd(const bf16 *d1, int cg_total, int cg0, long long nvox, int H, int W, const float *hw,
                            const float *hb, float *out, cudaStream_t s)
{
    head_fwd_kernel<<<nblk(nvox, 256), 256, 0, s>>>(d1, cg_total, cg0, nvox, H, W, hw, hb, out);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status launch_head_bwd(const bf16 *d1, int cg_total, int cg0, long long nvox, int H, int W, const float *out,
                            const float *target, const float *hw, float *g_hw, float *g_hb, bf16 *g_d1, double *loss,
                            cudaStream_t s)
{
    const unsigned blocks = (unsigned)std::min<long long>(4LL * sm_count(), std::max<long long>(1, nvox / 256));
    head_bwd_kernel<<<blocks, 256, 0, s>>>(d1, cg_total, cg0, nvox, H, W, out, target, hw, g_hw, g_hb, g_d1, loss);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status launch_adam(float *p, const float *g, float *m, float *v, int n, float lr, int step, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    adam_kernel<<<nblk(n, 256), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

}  // namespace gbsw

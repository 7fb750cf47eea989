// U-Net glue kernels: bias gradients, pooling / upsampling in the
// C8-blocked layout, the 1x1 head with the MSE loss, and Adam.
#include <algorithm>

#include "unet_ops.cuh"

namespace gbsw {

__device__ __forceinline__ size_t bidx(int zn, int cg_total, int cg, int H, int W, int y, int x)
{
    return ((((size_t)zn * cg_total + cg) * H + y) * W + x) * 8;
}

// ------------------------------------------------------------ bias grads
// db[co] += sum_v g[v, co] over a C8-blocked g (C channels at groups
// cg0 .. cg0 + C/8 - 1).  Thread t takes channel group t % (C/8) of the
// voxels t / (C/8), + 256 / (C/8), ...; the block then sums its threads'
// partials in a fixed order and adds one value per channel to db.
// Launch: block 256.
__global__ void __launch_bounds__(256)
bias_grad_kernel(const __nv_bfloat16 *__restrict__ g, int g_cg_total, int g_cg0, long long nvox, int H, int W, int C,
                 float *__restrict__ db)
{
    __shared__ float red[256][9];
    const int ng = C / 8;                 // 2, 4 or 8: divides 256
    const int lanes = 256 / ng;           // threads per channel group
    const int cb = threadIdx.x % ng, r = threadIdx.x / ng;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long v = (long long)blockIdx.x * lanes + r; v < nvox; v += (long long)gridDim.x * lanes) {
        const int xx = (int)(v % W);
        const int yy = (int)((v / W) % H);
        const int zn = (int)(v / ((long long)W * H));
        const uint4 pk = *reinterpret_cast<const uint4 *>(g + bidx(zn, g_cg_total, g_cg0 + cb, H, W, yy, xx));
        const __nv_bfloat16 *pb = reinterpret_cast<const __nv_bfloat16 *>(&pk);
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] += __bfloat162float(pb[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) red[threadIdx.x][q] = acc[q];
    __syncthreads();
    if (threadIdx.x < C) {
        const int c = threadIdx.x;
        float s = 0.0f;
        for (int l = 0; l < lanes; ++l) s += red[l * ng + c / 8][c % 8];
        atomicAdd(&db[c], s);
    }
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

gbsw_status launch_bias_grad(const bf16 *g, int g_cg_total, int g_cg0, long long nvox, int H, int W, int C,
                             float *db, cudaStream_t s)
{
    if (C % 8 || C > 64) return GBSW_ERR_ARG;
    const unsigned blocks = (unsigned)std::min<long long>(2LL * sm_count(), std::max<long long>(1, nvox / 256));
    bias_grad_kernel<<<blocks, 256, 0, s>>>(g, g_cg_total, g_cg0, nvox, H, W, C, db);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
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

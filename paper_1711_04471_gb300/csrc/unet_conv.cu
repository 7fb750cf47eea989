// tcgen05 implicit-GEMM 3x3x3 convolution (see unet_conv.cuh for the data
// layout and the pipeline), weight packing, and the operator-level C ABI
// used to check the kernel against the FP64 oracle.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "unet_conv.cuh"
#include "unet_internal.cuh"

namespace gbsw {

namespace {

constexpr int CONV_STAGES = 4;
constexpr int CONV_THREADS = 128;

__device__ __forceinline__ void set_status(int *status, int code) { atomicCAS(status, DEV_OK, code); }

template <int CIN, int COUT>
struct ConvSmem {
    static constexpr int A_BYTES = 128 * CIN * 2;
    static constexpr int B_BYTES = COUT * CIN * 2;
    static constexpr int STAGE = ((A_BYTES + B_BYTES + 1023) / 1024) * 1024;
    static constexpr int BAR_OFF = CONV_STAGES * STAGE;
    static constexpr int BYTES = BAR_OFF + 128 + 1024;  // barriers + TMEM slot, plus alignment slack
    static constexpr int TMEM_COLS = COUT < 32 ? 32 : COUT;
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(CONV_THREADS)
conv3d_tc_kernel(const __grid_constant__ CUtensorMap xmap, const __nv_bfloat16 *__restrict__ wpack,
                 const float *__restrict__ bias, __nv_bfloat16 *__restrict__ y, float *__restrict__ y_f32,
                 const __nv_bfloat16 *__restrict__ mask, ConvGeom g, int epi, int *status)
{
    using S = ConvSmem<CIN, COUT>;
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 256, "UMMA shape");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + S::BAR_OFF);
    uint64_t *empty = full + CONV_STAGES;
    uint64_t *done = empty + CONV_STAGES;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int t = blockIdx.x;
    const int tx = t % g.tiles_x;
    t /= g.tiles_x;
    const int ty = t % g.tiles_y;
    const int tz = t / g.tiles_y;
    const int x0 = tx * g.box_x, y0 = ty * g.box_y, z0 = tz * g.box_z;
    const bool multi = g.box_z > 1;  // tile of several planes (small planes)
    const int z = z0 % g.D;          // the plane of a single-plane tile

    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, S::TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < CONV_STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_mbar_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (threadIdx.x == 0) {
        // producer: one stage per valid tap
        int it = 0;
        for (int tap = 0; tap < 27; ++tap) {
            const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
            if (!multi && (z + dz < 0 || z + dz >= g.D)) continue;
            const int s = it % CONV_STAGES;
            if (it >= CONV_STAGES && !tc::mbar_wait(&empty[s], ((it / CONV_STAGES) - 1) & 1)) {
                set_status(status, DEV_TIMEOUT);
                break;
            }
            uint8_t *a = smem + s * S::STAGE;
            tc::mbar_arrive_expect_tx(&full[s], S::A_BYTES + S::B_BYTES);
            if (!multi) {
                tc::tma_load_5d(a, &xmap, &full[s], 0, x0 + dx, y0 + dy, 0, z0 + dz);
            } else {
                const int plane_bytes = g.box_x * g.box_y * 16;
                for (int zz = 0; zz < g.box_z; ++zz) {
                    const int zn = z0 + zz, zi = zn % g.D;
                    const int zsrc = (zn < g.NZ && zi + dz >= 0 && zi + dz < g.D) ? zn + dz : -1;
                    for (int cg = 0; cg < CIN / 8; ++cg)
                        tc::tma_load_5d(a + cg * 2048 + zz * plane_bytes, &xmap, &full[s], 0, x0 + dx, y0 + dy, cg,
                                        zsrc);
                }
            }
            tc::bulk_load(a + S::A_BYTES, wpack + (size_t)tap * COUT * CIN, S::B_BYTES, &full[s]);
            ++it;
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer
        constexpr uint32_t idesc = tc::idesc_bf16_f32(128, COUT);
        int it = 0;
        bool ok = true;
        for (int tap = 0; tap < 27 && ok; ++tap) {
            const int dz = tap / 9 - 1;
            if (!multi && (z + dz < 0 || z + dz >= g.D)) continue;
            const int s = it % CONV_STAGES;
            if (!tc::mbar_wait(&full[s], (it / CONV_STAGES) & 1)) {
                set_status(status, DEV_TIMEOUT);
                ok = false;
                break;
            }
            tc::fence_after_sync();
            const uint32_t a = tc::smem_u32(smem + s * S::STAGE);
            const uint32_t b = a + S::A_BYTES;
#pragma unroll
            for (int kc = 0; kc < CIN / 16; ++kc) {
                const uint64_t ad = tc::smem_desc(a + kc * 2 * 2048, 2048, 128);
                const uint64_t bd = tc::smem_desc(b + kc * 2 * COUT * 16, COUT * 16, 128);
                tc::umma_bf16(tmem, ad, bd, idesc, (it > 0 || kc > 0) ? 1u : 0u);
            }
            tc::umma_commit(&empty[s]);
            ++it;
        }
        tc::umma_commit(done);
    }

    // epilogue: thread = voxel (TMEM lane), 8 channels per TMEM load
    __syncwarp();  // lanes 0 of warps 0 and 1 rejoin after their producer / MMA roles
    const bool ready = tc::mbar_wait(done, 0);
    if (!ready && lane == 0) set_status(status, DEV_TIMEOUT);
    tc::fence_after_sync();
    const int m = warp * 32 + lane;
    const int plane = g.box_x * g.box_y;
    const int zn = z0 + m / plane, r = m % plane;
    const int yy = y0 + r / g.box_x, xx = x0 + r % g.box_x;
    const bool stored = zn < g.NZ;  // false only past the last plane of a multi-plane tile
#pragma unroll
    for (int cb = 0; cb < COUT / 8; ++cb) {
        float v[8];
        tc::tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + cb * 8, v);
        if (!ready || !stored) continue;
        if (epi == EPI_BIAS_RELU) {
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = fmaxf(v[q] + bias[cb * 8 + q], 0.0f);
        } else if (epi == EPI_MASK) {
            const uint4 mk = *reinterpret_cast<const uint4 *>(
                mask + ((((size_t)zn * g.mask_cg_total + g.mask_cg0 + cb) * g.H + yy) * g.W + xx) * 8);
            const __nv_bfloat16 *mb = reinterpret_cast<const __nv_bfloat16 *>(&mk);
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = __bfloat162float(mb[q]) > 0.0f ? v[q] : 0.0f;
        }
        if (y) {
            uint4 pk;
            __nv_bfloat162 *p2 = reinterpret_cast<__nv_bfloat162 *>(&pk);
#pragma unroll
            for (int q = 0; q < 4; ++q) p2[q] = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
            *reinterpret_cast<uint4 *>(y + ((((size_t)zn * g.out_cg_total + g.out_cg0 + cb) * g.H + yy) * g.W + xx) * 8) =
                pk;
        }
        if (y_f32) {
            float *o = y_f32 + (((size_t)zn * g.H + yy) * g.W + xx) * COUT + cb * 8;
#pragma unroll
            for (int q = 0; q < 8; ++q) o[q] = v[q];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, S::TMEM_COLS);
}

// ------------------------------------------------------------ weight grads
// Shared memory of wgrad_tc_kernel: a ring of stages, each holding the
// shifted x tiles of one group of TPG = 128 / CIN taps (the A operand, 128
// rows (tap, ci) of 2048-byte channel-group slabs, 32 KB) and the gz tile
// (B, COUT / 8 slabs).
template <int CIN, int COUT>
struct WgradSmem {
    static constexpr int TPG = 128 / CIN;                     // taps per MMA group
    static constexpr int NGROUPS = (27 + TPG - 1) / TPG;
    static constexpr int A_BYTES = 128 * 128 * 2;             // 16 slabs of 128 voxels x 16 B
    static constexpr int B_BYTES = COUT * 128 * 2;
    static constexpr int STAGE = A_BYTES + B_BYTES;           // a multiple of 2048
    static constexpr int STAGES = 4;
    static constexpr int BAR_OFF = STAGES * STAGE;
    static constexpr int BYTES = BAR_OFF + 128 + 1024;
    static constexpr int COLS_USED = NGROUPS * COUT;
    static constexpr int TMEM_COLS = COLS_USED <= 32 ? 32 : COLS_USED <= 64 ? 64 : COLS_USED <= 128 ? 128
                                   : COLS_USED <= 256 ? 256 : 512;
};

// dW[tap][co][ci] += sum over the voxels of tiles [t_begin, t_end) of
// gz[v][co] x[v + off(tap)][ci] (zero outside the sample), one CTA per
// chunk of tiles.  Per tile and tap group: thread 0 loads the group's
// shifted x tiles (the forward conv's TMA boxes; a plane whose tap leaves
// its sample, or past the last plane, is loaded from z = -1, all zero
// fill) and the gz tile into a stage; thread 32 issues 8 MMAs (M = 128
// rows (tap, ci), N = COUT, K = 16 voxels, both operands MN-major) into
// the group's TMEM columns; at the end the four warps add their 128 lanes
// (rows) of every group to dw with atomics.
template <int CIN, int COUT>
__global__ void __launch_bounds__(CONV_THREADS)
wgrad_tc_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap gmap, ConvGeom g,
                int tiles_per_cta, float *__restrict__ dw, int cin_store, int *status)
{
    using S = WgradSmem<CIN, COUT>;
    static_assert(CIN % 16 == 0 && 128 % CIN == 0 && COUT % 16 == 0 && S::COLS_USED <= 512, "wgrad shape");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = (uint64_t *)(smem + S::BAR_OFF);
    uint64_t *empty = full + S::STAGES;
    uint64_t *done = empty + S::STAGES;
    uint32_t *tmem_slot = (uint32_t *)(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = g.tiles_x * g.tiles_y * g.tiles_z;
    const int t_begin = blockIdx.x * tiles_per_cta;
    const int t_end = min(ntiles, t_begin + tiles_per_cta);
    const bool multi = g.box_z > 1;
    const int plane_bytes = g.box_x * g.box_y * 16;

    // rows of a partial last group read stale stage bytes: start them as zeros
    for (int q = threadIdx.x; q < S::STAGES * S::STAGE / 16; q += CONV_THREADS)
        reinterpret_cast<uint4 *>(smem)[q] = make_uint4(0, 0, 0, 0);
    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, S::TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < S::STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(done, 1);
        tc::fence_mbar_init();
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeros before any TMA / MMA access
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (threadIdx.x == 0) {
        // producer
        int it = 0;
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; ++t) {
            int tt = t;
            const int x0 = (tt % g.tiles_x) * g.box_x;
            tt /= g.tiles_x;
            const int y0 = (tt % g.tiles_y) * g.box_y;
            const int z0 = (tt / g.tiles_y) * g.box_z;
            for (int gi = 0; gi < S::NGROUPS; ++gi, ++it) {
                const int s = it % S::STAGES;
                if (it >= S::STAGES && !tc::mbar_wait(&empty[s], ((it / S::STAGES) - 1) & 1)) {
                    set_status(status, DEV_TIMEOUT);
                    ok = false;
                    break;
                }
                const int tap0 = gi * S::TPG;
                const int ntap = min(S::TPG, 27 - tap0);
                uint8_t *a = smem + s * S::STAGE;
                uint8_t *b = a + S::A_BYTES;
                tc::mbar_arrive_expect_tx(&full[s], ntap * CIN * 256 + COUT * 256);
                for (int q = 0; q < ntap; ++q) {
                    const int tap = tap0 + q;
                    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                    uint8_t *dst = a + q * (CIN / 8) * 2048;
                    if (!multi) {
                        const int z = z0 % g.D;
                        const int zsrc = (z + dz >= 0 && z + dz < g.D) ? z0 + dz : -1;
                        tc::tma_load_5d(dst, &xmap, &full[s], 0, x0 + dx, y0 + dy, 0, zsrc);
                    } else {
                        for (int zz = 0; zz < g.box_z; ++zz) {
                            const int zn = z0 + zz, zi = zn % g.D;
                            const int zsrc = (zn < g.NZ && zi + dz >= 0 && zi + dz < g.D) ? zn + dz : -1;
                            for (int cg = 0; cg < CIN / 8; ++cg)
                                tc::tma_load_5d(dst + cg * 2048 + zz * plane_bytes, &xmap, &full[s], 0, x0 + dx,
                                                y0 + dy, cg, zsrc);
                        }
                    }
                }
                if (!multi) {
                    tc::tma_load_5d(b, &gmap, &full[s], 0, x0, y0, 0, z0);
                } else {
                    for (int zz = 0; zz < g.box_z; ++zz) {
                        const int zn = z0 + zz;
                        for (int cg = 0; cg < COUT / 8; ++cg)
                            tc::tma_load_5d(b + cg * 2048 + zz * plane_bytes, &gmap, &full[s], 0, x0, y0, cg,
                                            zn < g.NZ ? zn : -1);
                    }
                }
            }
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer
        constexpr uint32_t idesc = tc::idesc_bf16_f32(128, COUT, true);
        int it = 0;
        bool ok = true;
        for (int t = t_begin; t < t_end && ok; ++t) {
            for (int gi = 0; gi < S::NGROUPS; ++gi, ++it) {
                const int s = it % S::STAGES;
                if (!tc::mbar_wait(&full[s], (it / S::STAGES) & 1)) {
                    set_status(status, DEV_TIMEOUT);
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t a = tc::smem_u32(smem + s * S::STAGE);
                const uint32_t b = a + S::A_BYTES;
#pragma unroll
                for (int kc = 0; kc < 8; ++kc) {
                    // K = 16 voxels per MMA: the start moves by 16 voxels x 16 B
                    const uint64_t ad = tc::smem_desc(a + kc * 256, 128, 2048);
                    const uint64_t bd = tc::smem_desc(b + kc * 256, 128, 2048);
                    tc::umma_bf16(tmem + gi * COUT, ad, bd, idesc, (t > t_begin || kc > 0) ? 1u : 0u);
                }
                tc::umma_commit(&empty[s]);
            }
        }
        tc::umma_commit(done);
    }

    // epilogue: lane = row (tap, ci) of a group, 8 output channels per load
    __syncwarp();
    const bool ready = t_end > t_begin && tc::mbar_wait(done, 0);
    if (!ready && t_end > t_begin && lane == 0) set_status(status, DEV_TIMEOUT);
    tc::fence_after_sync();
    const int row = warp * 32 + lane;
    const int ci = row % CIN;
#pragma unroll 1
    for (int gi = 0; gi < S::NGROUPS; ++gi) {
        const int tap = gi * S::TPG + row / CIN;
#pragma unroll
        for (int cb = 0; cb < COUT / 8; ++cb) {
            float v[8];
            tc::tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + gi * COUT + cb * 8, v);
            if (!ready || tap >= 27 || ci >= cin_store) continue;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                atomicAdd(&dw[((size_t)tap * COUT + cb * 8 + q) * cin_store + ci], v[q]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, S::TMEM_COLS);
}

// pack[tap][ci/8][co][ci%8] = w[tap][co][ci]   (forward), or with
// flip = 1 the weights of the backward-data convolution:
// pack[tap][co/8][ci][co%8] = w[26 - tap][co][ci].  The source holds
// cin_src <= cin input channels per (tap, co); the forward pack's channels
// ci >= cin_src are zero (a zero-padded input).
__global__ void conv_pack_kernel(const float *__restrict__ w, int cin_src, int cin, int cout, int flip,
                                 __nv_bfloat16 *__restrict__ pack)
{
    const int n = 27 * cin * cout;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int tap = q / (cin * cout);
    const int r = q % (cin * cout);
    const int co = r / cin, ci = r % cin;
    const float v = ci < cin_src ? w[((size_t)tap * cout + co) * cin_src + ci] : 0.0f;
    size_t dst;
    if (!flip) {
        dst = (((size_t)tap * (cin / 8) + ci / 8) * cout + co) * 8 + ci % 8;
    } else {
        const int tp = 26 - tap;  // the packed conv has Cin' = cout, Cout' = cin
        dst = (((size_t)tp * (cout / 8) + co / 8) * cin + ci) * 8 + co % 8;
    }
    pack[dst] = __float2bfloat16_rn(v);
}

// dense FP32 (zn, y, x, C) <-> C8-blocked BF16
__global__ void to_blocked_kernel(const float *__restrict__ src, int NZ, int H, int W, int C,
                                  __nv_bfloat16 *__restrict__ dst, int cg_total, int cg0)
{
    const long long n = (long long)NZ * H * W * C;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int c = (int)(q % C);
    long long v = q / C;
    const int x = (int)(v % W);
    v /= W;
    const int yy = (int)(v % H);
    const int zn = (int)(v / H);
    dst[((((size_t)zn * cg_total + cg0 + c / 8) * H + yy) * W + x) * 8 + c % 8] = __float2bfloat16_rn(src[q]);
}

__global__ void from_blocked_kernel(const __nv_bfloat16 *__restrict__ src, int NZ, int H, int W, int C, int cg_total,
                                    int cg0, float *__restrict__ dst)
{
    const long long n = (long long)NZ * H * W * C;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int c = (int)(q % C);
    long long v = q / C;
    const int x = (int)(v % W);
    v /= W;
    const int yy = (int)(v % H);
    const int zn = (int)(v / H);
    dst[q] = __bfloat162float(src[((((size_t)zn * cg_total + cg0 + c / 8) * H + yy) * W + x) * 8 + c % 8]);
}

using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                              const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn()
{
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeFn)p;
    });
    return fn;
}

template <int CIN, int COUT>
gbsw_status launch_conv_t(const ConvCall &c, cudaStream_t s)
{
    using S = ConvSmem<CIN, COUT>;
    static bool configured = false;
    if (!configured) {
        GBSW_CUDA_TRY(cudaFuncSetAttribute(conv3d_tc_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           S::BYTES));
        configured = true;
    }
    const int ntiles = c.geom.tiles_z * c.geom.tiles_y * c.geom.tiles_x;
    conv3d_tc_kernel<CIN, COUT><<<ntiles, CONV_THREADS, S::BYTES, s>>>(c.xmap, c.wpack, c.bias, c.y, c.y_f32, c.mask,
                                                                       c.geom, c.epi, c.status);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

template <int CIN, int COUT>
gbsw_status launch_wgrad_t(const WgradCall &c, cudaStream_t s)
{
    using S = WgradSmem<CIN, COUT>;
    static bool configured = false;
    if (!configured) {
        GBSW_CUDA_TRY(cudaFuncSetAttribute(wgrad_tc_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           S::BYTES));
        configured = true;
    }
    const int ntiles = c.geom.tiles_z * c.geom.tiles_y * c.geom.tiles_x;
    // one CTA per SM at most (the ring takes most of the shared memory); a
    // few tiles per CTA amortise the epilogue's atomics
    const int ctas = std::max(1, std::min(ntiles, sm_count()));
    const int per = ceil_div(ntiles, ctas);
    wgrad_tc_kernel<CIN, COUT><<<ceil_div(ntiles, per), CONV_THREADS, S::BYTES, s>>>(c.xmap, c.gmap, c.geom, per,
                                                                                     c.dw, c.cin_store, c.status);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

}  // namespace

// Geometry of a conv over a C8-blocked tensor of NZ planes of H x W voxels.
gbsw_status conv_geometry(int NZ, int D, int H, int W, ConvGeom *g)
{
    if (NZ < 1 || D < 1 || NZ % D != 0 || H < 1 || W < 1) return GBSW_ERR_ARG;
    int bx = W >= 128 ? 128 : W;
    if (bx < 1 || 128 % bx != 0 || W % bx != 0) return GBSW_ERR_ARG;  // W a power of two or a multiple of 128
    int by = 128 / bx, bz = 1;
    if (H < by) {
        // small planes: the tile spans bz planes of H rows; boxes of >= 256 bytes
        if (by % H != 0 || bx * H < 16) return GBSW_ERR_ARG;
        bz = by / H;
        by = H;
    } else if (H % by != 0) {
        return GBSW_ERR_ARG;
    }
    g->NZ = NZ;
    g->D = D;
    g->H = H;
    g->W = W;
    g->box_x = bx;
    g->box_y = by;
    g->box_z = bz;
    g->tiles_x = W / bx;
    g->tiles_y = H / by;
    g->tiles_z = (NZ + bz - 1) / bz;
    g->out_cg_total = g->out_cg0 = g->mask_cg_total = g->mask_cg0 = 0;
    return GBSW_OK;
}

// TMA map of a C8-blocked BF16 tensor with cg_total groups (all loaded).
gbsw_status conv_tensor_map(const __nv_bfloat16 *base, const ConvGeom &g, int cg_total, CUtensorMap *map)
{
    EncodeFn fn = encode_fn();
    if (!fn) return GBSW_ERR_CUDA;
    if (((uintptr_t)base & 15) != 0) return GBSW_ERR_ARG;
    const cuuint64_t dims[5] = {8, (cuuint64_t)g.W, (cuuint64_t)g.H, (cuuint64_t)cg_total, (cuuint64_t)g.NZ};
    const cuuint64_t strides[4] = {16, (cuuint64_t)g.W * 16, (cuuint64_t)g.H * g.W * 16,
                                   (cuuint64_t)cg_total * g.H * g.W * 16};
    // one box per tap (all channel groups), or per (plane, group) for multi-plane tiles
    const cuuint32_t box[5] = {8, (cuuint32_t)g.box_x, (cuuint32_t)g.box_y, g.box_z > 1 ? 1u : (cuuint32_t)cg_total,
                               1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, (void *)base, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GBSW_OK : GBSW_ERR_ARG;
}

gbsw_status launch_conv(int cin, int cout, const ConvCall &c, cudaStream_t s)
{
#define CONV_CASE(A, B) \
    if (cin == A && cout == B) return launch_conv_t<A, B>(c, s);
    CONV_CASE(16, 16)
    CONV_CASE(16, 32)
    CONV_CASE(16, 64)
    CONV_CASE(32, 16)
    CONV_CASE(32, 32)
    CONV_CASE(32, 64)
    CONV_CASE(64, 16)
    CONV_CASE(64, 32)
#undef CONV_CASE
    return GBSW_ERR_ARG;
}

gbsw_status launch_wgrad_tc(int cin, int cout, const WgradCall &c, cudaStream_t s)
{
#define WG_CASE(A, B) \
    if (cin == A && cout == B) return launch_wgrad_t<A, B>(c, s);
    WG_CASE(16, 16)
    WG_CASE(16, 32)
    WG_CASE(32, 16)
    WG_CASE(32, 32)
    WG_CASE(32, 64)
    WG_CASE(64, 16)
    WG_CASE(64, 32)
#undef WG_CASE
    return GBSW_ERR_ARG;
}

gbsw_status pack_weights(const float *w, int cin, int cout, int flip, __nv_bfloat16 *pack, cudaStream_t s)
{
    return pack_weights_padded(w, cin, cin, cout, flip, pack, s);
}

gbsw_status pack_weights_padded(const float *w, int cin_src, int cin, int cout, int flip, __nv_bfloat16 *pack,
                                cudaStream_t s)
{
    if (cin_src < 1 || cin_src > cin || (flip && cin_src != cin)) return GBSW_ERR_ARG;
    const int n = 27 * cin * cout;
    conv_pack_kernel<<<ceil_div(n, 256), 256, 0, s>>>(w, cin_src, cin, cout, flip, pack);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status to_blocked(const float *src, int NZ, int H, int W, int C, __nv_bfloat16 *dst, int cg_total, int cg0,
                       cudaStream_t s)
{
    const long long n = (long long)NZ * H * W * C;
    to_blocked_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, NZ, H, W, C, dst, cg_total, cg0);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status from_blocked(const __nv_bfloat16 *src, int NZ, int H, int W, int C, int cg_total, int cg0, float *dst,
                         cudaStream_t s)
{
    const long long n = (long long)NZ * H * W * C;
    from_blocked_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, NZ, H, W, C, cg_total, cg0, dst);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

}  // namespace gbsw

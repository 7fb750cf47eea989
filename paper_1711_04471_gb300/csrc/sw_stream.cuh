// Streaming, temporally blocked 2DSW kernel (Sec. 6.2 of arXiv:1711.04471:
// dyn -> shapiro -> update, fused over T time steps).
//
// Work decomposition.  A CTA of SWS_THREADS threads owns a strip of
// SWS_THREADS grid columns (one column per thread), of which the middle
// W = SWS_THREADS - 4T are written back (2 columns of halo per fused step
// on each side), and a segment of rows [r0, r1).  It marches up the strip
// one row per iteration.  Time level t -> t+1 is a pipeline stage: stage t
// receives a row of level t and emits the level-(t+1) row two rows below
// it (the y-radius of one step's dependency cone).  Stage t+1 consumes
// what stage t emitted in the previous iteration, so all stages share the
// three block barriers of an iteration; stage t works 3t rows behind
// stage 0 and the strip's output row trails the input row by 3T-1.
//
// Each thread keeps the y-neighbours of its own column in registers (the
// rolling window below); x-neighbours go through per-stage shared-memory
// line buffers.  Global memory is touched once per fused launch: level 0
// rows (eta, u, v, H) are loaded two rows ahead, level T rows are stored.
//
// One step on row n (level t -> t+1), with h = H + eta, wet = h > hmin:
//   u'(n)    = mask(u - g dt/dx (eta_e - eta_c))       (needs eta(x+1, n))
//   v'(n-1)  = mask(v - g dt/dy (eta(n) - eta(n-1)))
//   eta*(n-1)= eta - dt/dx (F_e - F_w) - dt/dy (G_n - G_s), upwind fluxes
//   eta+(n-2)= masked Shapiro filter of eta* (needs eta*(n-3..n-1))
#pragma once

#include <type_traits>

#include "sw_kernels.cuh"

namespace gbsw {

constexpr int SWS_THREADS = 128;   // strip width (threads = columns)
constexpr int SWS_PAD = 1;         // one guard column on each side of a line buffer
constexpr int SWS_LINE = SWS_THREADS + 2 * SWS_PAD;

// Rolling per-stage window of one column (registers).
struct SWStageRegs {
    float eta1, eta2;   // eta at rows n-1, n-2 (level t)
    float h1, h2, h3;   // h at rows n-1, n-2, n-3
    float H1, H2;       // still-water depth at rows n-1, n-2
    float v1;           // v (level t) at row n-1
    float vp2;          // v' at row n-2
    float up1, up2;     // u' at rows n-1, n-2
    float es2, es3;     // eta* at rows n-2, n-3
};

// A row of one column handed from a stage to the next (or loaded / stored).
struct SWRow {
    float eta, u, v, H;
};

// Per-stage shared line buffers.
struct SWStageLines {
    float eta[2][SWS_LINE];
    float h[4][SWS_LINE];
    float up[2][SWS_LINE];
    float es[2][SWS_LINE];
};

// Loads of the level-0 rows: through the read-only path when the inputs
// cannot change during the kernel (one fused launch), through L2 only
// (coherent across SMs) inside the persistent ensemble kernel, where other
// CTAs rewrite the buffers between levels.
enum class SWLoad { ReadOnly, L2 };

template <SWLoad LP>
__device__ __forceinline__ float sw_load(const float *ptr)
{
    if constexpr (LP == SWLoad::ReadOnly) return __ldg(ptr);
    else return __ldcg(ptr);
}

// One (strip, row segment) work item: T fused steps of the columns of
// strip `strip` (SWS_THREADS wide, W = SWS_THREADS - 4T written) for output
// rows [r0, r1).  All threads of the CTA must call it together.
template <int T, SWLoad LP>
__device__ __forceinline__ void sw_stream_tile(const SWDev &p, int strip, int r0, int r1,
                                               const float *__restrict__ H, const float *__restrict__ eta_in,
                                               const float *__restrict__ u_in, const float *__restrict__ v_in,
                                               float *__restrict__ eta_out, float *__restrict__ u_out,
                                               float *__restrict__ v_out, SWStageLines *lines)
{
    constexpr int W = SWS_THREADS - 4 * T;
    const int x = threadIdx.x;
    const int c = x + SWS_PAD;                      // index in a line buffer
    const int gi = strip * W - 2 * T + x;           // grid column of this thread
    const bool col_in = gi >= 0 && gi < p.nx;
    const bool owned = x >= 2 * T && x < 2 * T + W && col_in;
    const bool u_open = gi >= 0 && gi < p.nx - 1;   // not a wall face
    __syncthreads();  // the line buffers may still be in use by the previous work item

    // zero the guard columns once (they only feed discarded halo columns)
    if (x < 2 * T) {
        const int st = x >> 1;
        const int side = (x & 1) ? SWS_LINE - 1 : 0;
        for (int k = 0; k < 2; ++k) {
            lines[st].eta[k][side] = 0.0f;
            lines[st].up[k][side] = 0.0f;
            lines[st].es[k][side] = 0.0f;
        }
        for (int k = 0; k < 4; ++k) lines[st].h[k][side] = 0.0f;
    }

    const float hmin = p.hmin;
    SWStageRegs R[T];
    SWRow mail[T];  // mail[t]: level-(t+1) row emitted by stage t last iteration
#pragma unroll
    for (int t = 0; t < T; ++t) {
        R[t] = SWStageRegs{0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        mail[t] = SWRow{0, 0, 0, 0};
    }

    const long long extent = (long long)p.ny * p.pitch;  // elements of each field of this grid
    auto load_row = [&](int n) {
        SWRow r{0.0f, 0.0f, 0.0f, 0.0f};
        if (col_in && n >= 0 && n < p.ny && GBSW_INBOUNDS((long long)n * p.pitch + gi, extent, &g_sw_bounds)) {
            const size_t g = (size_t)n * p.pitch + gi;
            r.eta = sw_load<LP>(eta_in + g);
            r.u = sw_load<LP>(u_in + g);
            r.v = sw_load<LP>(v_in + g);
            r.H = sw_load<LP>(H + g);
        }
        return r;
    };

    // The ring slots of the line buffers repeat every 4 rows; the row loop
    // is unrolled by 4 so every slot index and the register window shift
    // are resolved at compile time.
    const int n_first = (r0 - 2 * T) & ~3;    // first level-0 row that matters, rounded down
    const int n_last = r1 - 1 + 3 * T - 1;    // iteration that emits output row r1-1
    SWRow pre0 = load_row(n_first), pre1 = load_row(n_first + 1);

    auto iteration = [&](auto phase, int n4) {
        constexpr int P = decltype(phase)::value;  // n & 3
        const int n = n4 + P;
        SWRow in[T];
        in[0] = pre0;
        pre0 = pre1;
        pre1 = load_row(n + 2);
#pragma unroll
        for (int t = 1; t < T; ++t) in[t] = mail[t - 1];

        // phase 1: publish eta and h of the incoming row of every stage
        float hn[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int s0 = (P - 3 * t) & 3;  // slot of row m = n - 3t
            hn[t] = __fadd_rn(in[t].H, in[t].eta);
            lines[t].eta[s0 & 1][c] = in[t].eta;
            lines[t].h[s0][c] = hn[t];
        }
        __syncthreads();
        // phase 2: momentum predictor u'(m), v'(m-1)
        float un[T], vn1[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int s0 = (P - 3 * t) & 3;
            const int m = n - 3 * t;
            const bool wc = hn[t] > hmin;
            float uv = 0.0f;
            if (u_open) {
                const float ee = lines[t].eta[s0 & 1][c + 1];
                const bool we = lines[t].h[s0][c + 1] > hmin;
                uv = sw_face_mask(sw_predict(in[t].u, p.gdt_dx, ee, in[t].eta), wc, we);
            }
            un[t] = uv;
            float vv = 0.0f;
            if (m - 1 >= 0 && m - 1 < p.ny - 1)
                vv = sw_face_mask(sw_predict(R[t].v1, p.gdt_dy, in[t].eta, R[t].eta1), R[t].h1 > hmin, wc);
            vn1[t] = vv;
            lines[t].up[s0 & 1][c] = uv;
        }
        __syncthreads();
        // phase 3: continuity eta*(m-1)
        float es1[T];
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int s1 = (P - 3 * t - 1) & 3;  // slot of row m-1
            const float uw = lines[t].up[s1 & 1][c - 1];
            const float he = lines[t].h[s1][c + 1], hw = lines[t].h[s1][c - 1];
            const float h1 = R[t].h1;
            const float fe = sw_upwind(R[t].up1, h1, he);
            const float fw = sw_upwind(uw, hw, h1);
            const float gn = sw_upwind(vn1[t], h1, hn[t]);
            const float gs = sw_upwind(R[t].vp2, R[t].h2, h1);
            es1[t] = __fsub_rn(R[t].eta1, __fmaf_rn(p.dt_dx, __fsub_rn(fe, fw), __fmul_rn(p.dt_dy, __fsub_rn(gn, gs))));
            lines[t].es[s1 & 1][c] = es1[t];
        }
        __syncthreads();
        // phase 4: Shapiro filter eta+(m-2), emit the level-(t+1) row m-2
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const int s2 = (P - 3 * t - 2) & 3;  // slot of row m-2
            const float es2 = R[t].es2;
            float out = es2;
            if (R[t].h2 > hmin) {
                const float we = lines[t].h[s2][c + 1] > hmin ? 1.0f : 0.0f;
                const float ww = lines[t].h[s2][c - 1] > hmin ? 1.0f : 0.0f;
                const float wn = R[t].h1 > hmin ? 1.0f : 0.0f;
                const float ws = R[t].h3 > hmin ? 1.0f : 0.0f;
                const float ee = lines[t].es[s2 & 1][c + 1];
                const float ew = lines[t].es[s2 & 1][c - 1];
                const float cnt = (we + ww) + (wn + ws);  // small integers: exact
                const float sum = __fadd_rn(__fadd_rn(__fmul_rn(we, ee), __fmul_rn(ww, ew)),
                                            __fadd_rn(__fmul_rn(wn, es1[t]), __fmul_rn(ws, R[t].es3)));
                out = __fmaf_rn(p.q, sum, __fmul_rn(__fsub_rn(1.0f, __fmul_rn(p.q, cnt)), es2));
            }
            mail[t] = SWRow{out, R[t].up2, R[t].vp2, R[t].H2};
            // roll the window
            SWStageRegs &r = R[t];
            r.eta2 = r.eta1;
            r.eta1 = in[t].eta;
            r.h3 = r.h2;
            r.h2 = r.h1;
            r.h1 = hn[t];
            r.H2 = r.H1;
            r.H1 = in[t].H;
            r.v1 = in[t].v;
            r.vp2 = vn1[t];
            r.up2 = r.up1;
            r.up1 = un[t];
            r.es3 = r.es2;
            r.es2 = es1[t];
        }
        // the last stage's row is final: level T at row n - 3T + 1
        const int out_row = n - 3 * T + 1;
        if (owned && out_row >= r0 && out_row < r1 &&
            GBSW_INBOUNDS((long long)out_row * p.pitch + gi, extent, &g_sw_bounds)) {
            const size_t g = (size_t)out_row * p.pitch + gi;
            eta_out[g] = mail[T - 1].eta;
            u_out[g] = mail[T - 1].u;
            v_out[g] = mail[T - 1].v;
        }
    };

#pragma unroll 1
    for (int n4 = n_first; n4 <= n_last; n4 += 4) {
        iteration(std::integral_constant<int, 0>{}, n4);
        iteration(std::integral_constant<int, 1>{}, n4);
        iteration(std::integral_constant<int, 2>{}, n4);
        iteration(std::integral_constant<int, 3>{}, n4);
    }
}

// One fused launch of depth T over a single grid.  grid (strips, segments),
// block SWS_THREADS; rows_per_cta rows per segment.
template <int T>
__global__ void __launch_bounds__(SWS_THREADS)
sw_stream_kernel(SWDev p, int rows_per_cta, const float *__restrict__ H, const float *__restrict__ eta_in,
                 const float *__restrict__ u_in, const float *__restrict__ v_in, float *__restrict__ eta_out,
                 float *__restrict__ u_out, float *__restrict__ v_out)
{
    __shared__ SWStageLines lines[T];
    const int r0 = blockIdx.y * rows_per_cta;
    if (r0 >= p.ny) return;
    const int r1 = min(p.ny, r0 + rows_per_cta);
    sw_stream_tile<T, SWLoad::ReadOnly>(p, blockIdx.x, r0, r1, H, eta_in, u_in, v_in, eta_out, u_out, v_out, lines);
}

}  // namespace gbsw

// Tile kernel of the 2DSW step for grids that stay in L2 (Sec. 6.2 of
// arXiv:1711.04471: dyn -> shapiro -> update, T steps fused per launch).
//
// A CTA loads a tile of SWT_W x SWT_H cells plus a halo of 2T cells on
// every side (the dependency radius of one step is 2 cells) into shared
// memory, advances the whole tile T steps there, and writes back the
// middle SWT_W x SWT_H cells.  Each step is four barrier-separated phases
// over the tile: depth h, momentum predictor u', v' (in place of u, v),
// continuity eta*, masked Shapiro filter (in place of eta).  Cells past a
// tile edge are not read (the results there are discarded halo); cells
// outside the grid are loaded as H = eta = u = v = 0 and stay so, exactly
// as in the streaming kernel.  Every operation is the streaming kernel's,
// rounded in the same order (explicit round-to-nearest intrinsics), so the
// two kernels give bitwise the same state.
//
// Compared with the streaming kernel, a launch has no row-by-row pipeline:
// its latency is one load, 4T short phases and one store, which is what
// the small grids of the paper (500^2 .. 2000^2, a few MB) need.
#pragma once

#include "sw_kernels.cuh"

namespace gbsw {

constexpr int SWT_W = 32, SWT_H = 32;   // written cells of a tile
constexpr int SWT_THREADS = 1024;  // about two cells per thread and phase: the phases are short, latency-bound loops
constexpr int SWT_MAX_T = 3;             // 6 arrays of (32 + 4T)^2 floats fit the 48 KB static limit

template <int T>
__global__ void __launch_bounds__(SWT_THREADS)
sw_tile_kernel(SWDev p, const float *__restrict__ H, const float *__restrict__ eta_in, const float *__restrict__ u_in,
               const float *__restrict__ v_in, float *__restrict__ eta_out, float *__restrict__ u_out,
               float *__restrict__ v_out)
{
    constexpr int HALO = 2 * T;
    constexpr int LW = SWT_W + 2 * HALO, LH = SWT_H + 2 * HALO, NC = LW * LH;
    __shared__ float e[NC], uu[NC], vv[NC], HH[NC], hh[NC], es[NC];
    const int x0 = blockIdx.x * SWT_W - HALO, y0 = blockIdx.y * SWT_H - HALO;
    const float hmin = p.hmin;

    for (int q = threadIdx.x; q < NC; q += SWT_THREADS) {
        const int lx = q % LW, ly = q / LW, gx = x0 + lx, gy = y0 + ly;
        float a = 0.0f, b = 0.0f, c = 0.0f, d = 0.0f;
        if (gx >= 0 && gx < p.nx && gy >= 0 && gy < p.ny &&
            GBSW_INBOUNDS((long long)gy * p.pitch + gx, (long long)p.ny * p.pitch, &g_sw_bounds)) {
            const size_t g = (size_t)gy * p.pitch + gx;
            a = __ldg(eta_in + g);
            b = __ldg(u_in + g);
            c = __ldg(v_in + g);
            d = __ldg(H + g);
        }
        e[q] = a;
        uu[q] = b;
        vv[q] = c;
        HH[q] = d;
    }
    __syncthreads();
#pragma unroll 1
    for (int t = 0; t < T; ++t) {
        for (int q = threadIdx.x; q < NC; q += SWT_THREADS) hh[q] = __fadd_rn(HH[q], e[q]);
        __syncthreads();
        // momentum predictor of the east and north faces of each cell
        for (int q = threadIdx.x; q < NC; q += SWT_THREADS) {
            const int lx = q % LW, ly = q / LW, gx = x0 + lx, gy = y0 + ly;
            const bool wc = hh[q] > hmin;
            float un = 0.0f, vn = 0.0f;
            if (lx + 1 < LW && gx >= 0 && gx < p.nx - 1)
                un = sw_face_mask(sw_predict(uu[q], p.gdt_dx, e[q + 1], e[q]), wc, hh[q + 1] > hmin);
            if (ly + 1 < LH && gy >= 0 && gy < p.ny - 1)
                vn = sw_face_mask(sw_predict(vv[q], p.gdt_dy, e[q + LW], e[q]), wc, hh[q + LW] > hmin);
            uu[q] = un;
            vv[q] = vn;
        }
        __syncthreads();
        // continuity with upwind face fluxes
        for (int q = threadIdx.x; q < NC; q += SWT_THREADS) {
            const int lx = q % LW, ly = q / LW;
            float out = e[q];
            if (lx > 0 && lx + 1 < LW && ly > 0 && ly + 1 < LH) {
                const float h1 = hh[q];
                const float fe = sw_upwind(uu[q], h1, hh[q + 1]);
                const float fw = sw_upwind(uu[q - 1], hh[q - 1], h1);
                const float gn = sw_upwind(vv[q], h1, hh[q + LW]);
                const float gs = sw_upwind(vv[q - LW], hh[q - LW], h1);
                out = __fsub_rn(e[q], __fmaf_rn(p.dt_dx, __fsub_rn(fe, fw), __fmul_rn(p.dt_dy, __fsub_rn(gn, gs))));
            }
            es[q] = out;
        }
        __syncthreads();
        // masked Shapiro filter on wet cells
        for (int q = threadIdx.x; q < NC; q += SWT_THREADS) {
            const int lx = q % LW, ly = q / LW;
            float out = es[q];
            if (lx > 0 && lx + 1 < LW && ly > 0 && ly + 1 < LH && hh[q] > hmin) {
                const float we = hh[q + 1] > hmin ? 1.0f : 0.0f;
                const float ww = hh[q - 1] > hmin ? 1.0f : 0.0f;
                const float wn = hh[q + LW] > hmin ? 1.0f : 0.0f;
                const float ws = hh[q - LW] > hmin ? 1.0f : 0.0f;
                const float cnt = (we + ww) + (wn + ws);  // small integers: exact
                const float sum = __fadd_rn(__fadd_rn(__fmul_rn(we, es[q + 1]), __fmul_rn(ww, es[q - 1])),
                                            __fadd_rn(__fmul_rn(wn, es[q + LW]), __fmul_rn(ws, es[q - LW])));
                out = __fmaf_rn(p.q, sum, __fmul_rn(__fsub_rn(1.0f, __fmul_rn(p.q, cnt)), es[q]));
            }
            e[q] = out;
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < SWT_W * SWT_H; q += SWT_THREADS) {
        const int lx = HALO + q % SWT_W, ly = HALO + q / SWT_W, gx = x0 + lx, gy = y0 + ly;
        if (gx < p.nx && gy < p.ny &&
            GBSW_INBOUNDS((long long)gy * p.pitch + gx, (long long)p.ny * p.pitch, &g_sw_bounds)) {
            const size_t g = (size_t)gy * p.pitch + gx;
            const int c = ly * LW + lx;
            eta_out[g] = e[c];
            u_out[g] = uu[c];
            v_out[g] = vv[c];
        }
    }
}

}  // namespace gbsw

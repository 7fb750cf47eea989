// Tile kernel of the 2DSW step for grids that stay in L2 (Sec. 6.2 of
// arXiv:1711.04471: dyn -> shapiro -> update, T steps fused per launch).
//
// A CTA loads a tile of SWT_W x SWT_H cells plus a halo of 2T cells on
// every side (the dependency radius of one step is 2 cells) into shared
// memory, advances the whole tile T steps there, and writes back the
// middle SWT_W x SWT_H cells.  Each step is three barrier-separated
// phases over the tile: momentum predictor u', v'; continuity eta*;
// masked Shapiro filter, which also forms the next step's depth h (in the
// other of two h buffers, since this phase still reads the current one).
// A thread keeps its own cells' values in registers (H never leaves
// them); shared memory holds only what the neighbours read.  Cells past a
// tile edge are not read (the results there are discarded halo); cells
// outside the grid are loaded as H = eta = u = v = 0 and stay so, exactly
// as in the streaming kernel.  Every operation is the streaming kernel's,
// rounded in the same order (explicit round-to-nearest intrinsics), so the
// two kernels give bitwise the same state.
//
// Compared with the streaming kernel, a launch has no row-by-row pipeline:
// its latency is one load, 3T short phases and one store, which is what
// the small grids of the paper (500^2 .. 2000^2, a few MB) need.
#pragma once

#include "sw_kernels.cuh"

namespace gbsw {

constexpr int SWT_W = 32, SWT_H = 32;   // written cells of a tile
constexpr int SWT_THREADS = 1024;  // about two cells per thread and phase: the phases are short, latency-bound loops
constexpr int SWT_MAX_T = 3;             // 6 arrays of (32 + 4T)^2 floats fit the 48 KB static limit

// A load of state that the previous launch wrote: an ordered load (it may
// not be moved above griddepcontrol.wait, as a load through the read-only
// path may) that bypasses L1.
__device__ __forceinline__ float ld_state(const float *ptr)
{
    float v;
    asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(ptr) : "memory");
    return v;
}

template <int T>
__global__ void __launch_bounds__(SWT_THREADS, 2)
sw_tile_kernel(SWDev p, const float *__restrict__ H, const float *__restrict__ eta_in, const float *__restrict__ u_in,
               const float *__restrict__ v_in, float *__restrict__ eta_out, float *__restrict__ u_out,
               float *__restrict__ v_out)
{
    constexpr int HALO = 2 * T;
    constexpr int LW = SWT_W + 2 * HALO, LH = SWT_H + 2 * HALO, NC = LW * LH;
    constexpr int PER = (NC + SWT_THREADS - 1) / SWT_THREADS;  // cells per thread (2 for T <= 3)
    // neighbours' values only: each thread keeps its own cells' values in registers
    __shared__ float e[NC], uu[NC], vv[NC], hh2[2][NC], es[NC];  // depth double-buffered by step
    const int x0 = blockIdx.x * SWT_W - HALO, y0 = blockIdx.y * SWT_H - HALO;
    const float hmin = p.hmin;

    float re[PER], ru[PER], rv[PER], rH[PER], rh[PER], rs[PER];
    int lx[PER], ly[PER];
    bool act[PER], in[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = threadIdx.x + k * SWT_THREADS;
        act[k] = q < NC;
        lx[k] = q % LW;
        ly[k] = q / LW;
        const int gx = x0 + lx[k], gy = y0 + ly[k];
        in[k] = act[k] && gx >= 0 && gx < p.nx && gy >= 0 && gy < p.ny &&
                GBSW_INBOUNDS((long long)gy * p.pitch + gx, (long long)p.ny * p.pitch, &g_sw_bounds);
        // H is written by no step kernel, so it may be read before the wait below
        rH[k] = in[k] ? __ldg(H + ((size_t)gy * p.pitch + gx)) : 0.0f;
    }
    // Programmatic dependent launch: when this launch follows another tile
    // launch with that dependency, its blocks may be scheduled while the
    // previous launch drains, and they read no state before the previous
    // launch has completed and its writes are visible.  The next launch may
    // be scheduled as soon as every block of this one has started.  Both
    // are no-ops for a launch without that dependency.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int gx = x0 + lx[k], gy = y0 + ly[k];
        float a = 0.0f, b = 0.0f, c = 0.0f;
        if (in[k]) {
            const size_t g = (size_t)gy * p.pitch + gx;
            a = ld_state(eta_in + g);
            b = ld_state(u_in + g);
            c = ld_state(v_in + g);
        }
        re[k] = a;
        ru[k] = b;
        rv[k] = c;
        rs[k] = 0.0f;
        // depth of the first step, and the fields the neighbours read
        rh[k] = __fadd_rn(rH[k], re[k]);
        if (act[k]) {
            hh2[0][threadIdx.x + k * SWT_THREADS] = rh[k];
            e[threadIdx.x + k * SWT_THREADS] = re[k];
        }
    }
    __syncthreads();
    // The step loop is unrolled so that each step's pair of h buffers is
    // fixed at compile time.  The rolled loop (buffer picked from t at run
    // time) gave states that differed from the streaming kernel at T = 3 in
    // the bitwise tiling tests; the cause was not found, and the unrolled
    // form matches bit for bit.
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const float *hh = hh2[t & 1];
        // Rows that can still reach the written block: those within 2 (T - t)
        // of it for the predictor, one fewer per later phase.  The other
        // rows hold discarded halo, so they are skipped.
        const int B_LO = 2 * t, C_LO = 2 * t + 1, D_LO = 2 * t + 2;  // constants once the loop is unrolled
        // momentum predictor of the east and north faces of each cell
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            if (!act[k] || ly[k] < B_LO || ly[k] >= LH - B_LO) continue;
            const int q = threadIdx.x + k * SWT_THREADS;
            const int gx = x0 + lx[k], gy = y0 + ly[k];
            const bool wc = rh[k] > hmin;
            float un = 0.0f, vn = 0.0f;
            if (lx[k] + 1 < LW && gx >= 0 && gx < p.nx - 1)
                un = sw_face_mask(sw_predict(ru[k], p.gdt_dx, e[q + 1], re[k]), wc, hh[q + 1] > hmin);
            if (ly[k] + 1 < LH && gy >= 0 && gy < p.ny - 1)
                vn = sw_face_mask(sw_predict(rv[k], p.gdt_dy, e[q + LW], re[k]), wc, hh[q + LW] > hmin);
            ru[k] = un;
            rv[k] = vn;
            uu[q] = un;
            vv[q] = vn;
        }
        __syncthreads();
        // continuity with upwind face fluxes
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            if (!act[k] || ly[k] < C_LO || ly[k] >= LH - C_LO) continue;
            const int q = threadIdx.x + k * SWT_THREADS;
            float out = re[k];
            if (lx[k] > 0 && lx[k] + 1 < LW && ly[k] > 0 && ly[k] + 1 < LH) {
                const float h1 = rh[k];
                const float fe = sw_upwind(ru[k], h1, hh[q + 1]);
                const float fw = sw_upwind(uu[q - 1], hh[q - 1], h1);
                const float gn = sw_upwind(rv[k], h1, hh[q + LW]);
                const float gs = sw_upwind(vv[q - LW], hh[q - LW], h1);
                out = __fsub_rn(re[k], __fmaf_rn(p.dt_dx, __fsub_rn(fe, fw), __fmul_rn(p.dt_dy, __fsub_rn(gn, gs))));
            }
            rs[k] = out;
            es[q] = out;
        }
        __syncthreads();
        // masked Shapiro filter on wet cells
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            if (!act[k] || ly[k] < D_LO || ly[k] >= LH - D_LO) continue;
            const int q = threadIdx.x + k * SWT_THREADS;
            float out = rs[k];
            if (lx[k] > 0 && lx[k] + 1 < LW && ly[k] > 0 && ly[k] + 1 < LH && rh[k] > hmin) {
                const float we = hh[q + 1] > hmin ? 1.0f : 0.0f;
                const float ww = hh[q - 1] > hmin ? 1.0f : 0.0f;
                const float wn = hh[q + LW] > hmin ? 1.0f : 0.0f;
                const float ws = hh[q - LW] > hmin ? 1.0f : 0.0f;
                const float cnt = (we + ww) + (wn + ws);  // small integers: exact
                const float sum = __fadd_rn(__fadd_rn(__fmul_rn(we, es[q + 1]), __fmul_rn(ww, es[q - 1])),
                                            __fadd_rn(__fmul_rn(wn, es[q + LW]), __fmul_rn(ws, es[q - LW])));
                out = __fmaf_rn(p.q, sum, __fmul_rn(__fsub_rn(1.0f, __fmul_rn(p.q, cnt)), rs[k]));
            }
            re[k] = out;
            if (t + 1 < T) {
                // the next step's depth goes to the other buffer: this phase still reads hh
                rh[k] = __fadd_rn(rH[k], out);
                hh2[(t + 1) & 1][q] = rh[k];
                e[q] = out;
            }
        }
        if (t + 1 < T) __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        if (!act[k] || lx[k] < HALO || lx[k] >= HALO + SWT_W || ly[k] < HALO || ly[k] >= HALO + SWT_H) continue;
        const int gx = x0 + lx[k], gy = y0 + ly[k];
        if (gx < p.nx && gy < p.ny &&
            GBSW_INBOUNDS((long long)gy * p.pitch + gx, (long long)p.ny * p.pitch, &g_sw_bounds)) {
            const size_t g = (size_t)gy * p.pitch + gx;
            eta_out[g] = re[k];
            u_out[g] = ru[k];
            v_out[g] = rv[k];
        }
    }
}

}  // namespace gbsw

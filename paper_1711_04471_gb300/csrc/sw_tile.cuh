// Tile kernel of the 2DSW step for grids that stay in L2 (Sec. 6.2 of
// arXiv:1711.04471: dyn -> shapiro -> update, T steps fused per launch).
//
// A CTA loads a tile of SWT_W columns x th rows (th = SWT_H unless the
// launch picks another height, so that the CTAs spread evenly over the
// SMs) plus a halo of 2T cells on every side (the dependency radius of one
// step is 2 cells) into shared memory, advances the whole tile T steps
// there, and writes back the middle SWT_W x th cells.  Each step is three barrier-separated
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

constexpr int SWT_W = 32;           // written columns of a tile
constexpr int SWT_H = 32;           // written rows of a tile unless the launch asks for another height
constexpr int SWT_THREADS = 1024;   // about two cells per thread and phase: the phases are short, latency-bound loops
constexpr int SWT_PER = 2;          // cells per thread
constexpr int SWT_NC_MAX = SWT_PER * SWT_THREADS;  // cells of a tile with its halo: 6 arrays of them fill the 48 KB static limit
constexpr int SWT_MAX_T = 3;        // a 32 x 32 tile with its halo fits up to T = 3

// Most written rows of a tile of depth T: (SWT_W + 4T)(rows + 4T) <= SWT_NC_MAX
// (52, 43 and 34 rows for T = 1, 2, 3).
constexpr int swt_max_rows(int T) { return SWT_NC_MAX / (SWT_W + 4 * T) - 4 * T; }
static_assert(swt_max_rows(SWT_MAX_T) >= SWT_H, "the default tile must fit at the deepest fusion");

// Row flags of the tile kernel of depth T as a table: the 9 bits at 9d are
// those of a row d rows from the tile's nearer top or bottom edge (d = 0 ..
// 2T): bit 3t + ph for every phase ph of step t with 2t + ph <= d.
__host__ __device__ constexpr unsigned long long swt_row_bits(int T)
{
    unsigned long long tab = 0;
    for (int d = 0; d <= 2 * T; ++d)
        for (int t = 0; t < T; ++t)
            for (int ph = 0; ph < 3; ++ph)
                if (2 * t + ph <= d) tab |= 1ull << (9 * d + 3 * t + ph);
    return tab;
}

// A load of state that the previous launch wrote: an ordered load (it may
// not be moved above griddepcontrol.wait, as a load through the read-only
// path may) that bypasses L1.
__device__ __forceinline__ float ld_state(const float *ptr)
{
    float v;
    asm volatile("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(ptr) : "memory");
    return v;
}

// th: written rows of a tile (2 .. swt_max_rows(T), checked by the host);
// grid = (ceil(nx / SWT_W), ceil(ny / th)).
template <int T>
__global__ void __launch_bounds__(SWT_THREADS, 2)
sw_tile_kernel(SWDev p, int th, const float *__restrict__ H, const float *__restrict__ eta_in,
               const float *__restrict__ u_in, const float *__restrict__ v_in, float *__restrict__ eta_out,
               float *__restrict__ u_out, float *__restrict__ v_out)
{
    constexpr int HALO = 2 * T;
    constexpr int LW = SWT_W + 2 * HALO;  // the row stride of the shared arrays stays a constant
    constexpr int PER = SWT_PER;
    const int LH = th + 2 * HALO, NC = LW * LH;  // NC <= SWT_NC_MAX
    // neighbours' values only: each thread keeps its own cells' values in registers
    __shared__ float e[SWT_NC_MAX], uu[SWT_NC_MAX], vv[SWT_NC_MAX], hh2[2][SWT_NC_MAX],
        es[SWT_NC_MAX];  // depth double-buffered by step
    const int x0 = blockIdx.x * SWT_W - HALO, y0 = blockIdx.y * th - HALO;
    const float hmin = p.hmin;

    // Per-cell flags, fixed for the launch: bit 3t + ph (t < T; ph = 0
    // predictor, 1 continuity, 2 Shapiro) when the cell's row can still
    // reach the written block in that phase (rows within 2(T - t) of it for
    // the predictor, one fewer per later phase, i.e. at least 2t + ph rows
    // from the tile's top and bottom edges; the other rows hold discarded
    // halo and are skipped), and the bits below.
    constexpr unsigned F_EAST = 1u << 9;    // east face inside the grid and the tile
    constexpr unsigned F_NORTH = 1u << 10;  // north face inside the grid and the tile
    constexpr unsigned F_INNER = 1u << 11;  // not on the tile's edge: all four neighbours are in the tile
    constexpr unsigned F_STORE = 1u << 12;  // written back (inside the written block and the grid)
    constexpr unsigned F_LOAD = 1u << 13;   // inside the grid: loaded (else H = eta = u = v = 0)
    constexpr unsigned F_CELL = 1u << 14;   // a cell of the tile (q < NC)
    constexpr unsigned long long ROWS = swt_row_bits(T);
    float re[PER], ru[PER], rv[PER], rH[PER], rh[PER], rs[PER];
    unsigned m[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = threadIdx.x + k * SWT_THREADS;
        const int lx = q % LW, ly = q / LW;
        const int gx = x0 + lx, gy = y0 + ly;
        unsigned f = 0;
        if (q < NC) {
            const int dy = min(ly, LH - 1 - ly);  // rows to the nearer of the tile's top and bottom edges
            f |= F_CELL | (unsigned)((ROWS >> (9 * min(dy, 2 * T))) & 0x1ffull);
            if (lx + 1 < LW && gx >= 0 && gx < p.nx - 1) f |= F_EAST;
            if (ly + 1 < LH && gy >= 0 && gy < p.ny - 1) f |= F_NORTH;
            if (lx > 0 && lx + 1 < LW && dy > 0) f |= F_INNER;
            const bool in_grid = gx >= 0 && gx < p.nx && gy >= 0 && gy < p.ny &&
                                 GBSW_INBOUNDS((long long)gy * p.pitch + gx, (long long)p.ny * p.pitch, &g_sw_bounds);
            if (in_grid) f |= F_LOAD;
            if (in_grid && lx >= HALO && lx < HALO + SWT_W && ly >= HALO && ly < HALO + th) f |= F_STORE;
        }
        m[k] = f;
        // H is written by no step kernel, so it may be read before the wait below
        rH[k] = (f & F_LOAD) ? __ldg(H + ((size_t)gy * p.pitch + gx)) : 0.0f;
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
        const int q = threadIdx.x + k * SWT_THREADS;
        float a = 0.0f, b = 0.0f, c = 0.0f;
        if (m[k] & F_LOAD) {
            const size_t g = (size_t)(y0 + q / LW) * p.pitch + (x0 + q % LW);
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
        if (m[k] & F_CELL) {
            hh2[0][q] = rh[k];
            e[q] = re[k];
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
        const unsigned F_B = 1u << (3 * t), F_C = 1u << (3 * t + 1), F_D = 1u << (3 * t + 2);
        // momentum predictor of the east and north faces of each cell
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            if (!(m[k] & F_B)) continue;
            const int q = threadIdx.x + k * SWT_THREADS;
            const bool wc = rh[k] > hmin;
            float un = 0.0f, vn = 0.0f;
            if (m[k] & F_EAST)
                un = sw_face_mask(sw_predict(ru[k], p.gdt_dx, e[q + 1], re[k]), wc, hh[q + 1] > hmin);
            if (m[k] & F_NORTH)
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
            if (!(m[k] & F_C)) continue;
            const int q = threadIdx.x + k * SWT_THREADS;
            float out = re[k];
            if (m[k] & F_INNER) {
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
            if (!(m[k] & F_D)) continue;
            const int q = threadIdx.x + k * SWT_THREADS;
            float out = rs[k];
            if ((m[k] & F_INNER) && rh[k] > hmin) {
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
        if (!(m[k] & F_STORE)) continue;
        const int q = threadIdx.x + k * SWT_THREADS;
        const size_t g = (size_t)(y0 + q / LW) * p.pitch + (x0 + q % LW);
        eta_out[g] = re[k];
        u_out[g] = ru[k];
        v_out[g] = rv[k];
    }
}

}  // namespace gbsw

// Red-black SOR pressure solve ("press", Sec. 6.3.1 of arXiv:1711.04471)
// with an FP64 residual norm and a device-side convergence test: one solve
// is one launch of a CUDA graph whose while-node repeats
// [m SOR iterations, fold, FP64 residual, test] until ||b - A p|| <= tol ||b||
// or max_iter, with no host round trip.  With predicted checks (the UFLES
// step) the body is a chunk of iterations followed by a check node that
// runs only when the convergence rate puts the tolerance within reach.
//
// FP64 runs at a small fraction of the FP32 rate on this GPU, so the check
// is arranged to spend few FP64 operations per cell: the FP32 correction is
// folded into the FP64 base once per check (2 operations per cell), the
// residual is then a plain FP64 stencil of the base (no per-neighbour
// conversion), and ||b||^2 is formed once per solve.
#include <math.h>
#include <stdlib.h>

#include <algorithm>

#include "poisson.cuh"

namespace gbsw {

// Out-of-range index count of the bounds-checked debug build.
static __device__ unsigned g_sor_bounds;

unsigned long long take_bounds_poisson()
{
    unsigned h = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&h, g_sor_bounds, sizeof(h)) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_sor_bounds, &zero, sizeof(zero));
    return h;
}

__device__ __forceinline__ long long pidx(const PDims &d, int i, int j, int k)
{
    return (long long)k * d.plane + (long long)j * d.pitch + i;
}

// Slot of cell (i, j, k) in the array of its colour.
__device__ __forceinline__ long long cidx(const PDims &d, int i, int j, int k)
{
    return (long long)k * d.cplane + (long long)j * d.cpitch + SOR_SLOT0 + ((i - 1) >> 1);
}


// One colour half-sweep over cells with (i + j + k) % 2 == colour.  A
// thread owns the cells of that colour at slots s0 .. s0+3 of row j on
// planes SOR_KZ blockIdx.z + 1 .. SOR_KZ blockIdx.z + SOR_KZ.  Rows of a
// whole number of 32-group warps (FLAT = false): block = 32 groups of
// SOR_THREADS / 32 consecutive rows, so a warp holds one row (its colour
// parity q is warp-uniform).  Other rows (FLAT = true): thread t of a block
// takes group t mod G of row t / G (G = groups per row), so no lane idles
// at the end of a row; q may then differ inside a warp.
// Every access of a plane is one 16-byte vector (own correction, residual,
// the other colour's y and z neighbours and its four x neighbours) plus
// one word (the fifth x neighbour, the other colour's slot s0 - 1 or
// s0 + 4).  In-plane offsets are 32-bit (a colour plane holds fewer than
// 2^31 words for every accepted size).
// The per-cell arithmetic is the SOR update
//   e <- e + omega ((sum of the six neighbours - dx^2 r) / d_c - e)
// with the neighbour sum associated as (x pair + y pair) + z pair and the
// division correctly rounded (sor_div).  d_c is 6 inside, 5 on the ground
// and lid planes, one less at i = 1 and one more at i = nx (the entry
// points require nx, nz >= 2).
// Slots beyond the last cell of a row are pad words: they are written 0.
// FIRST: first iteration after a residual check; the correction restarts
// from 0 (the fold before the check has zeroed it), so the first red
// half-sweep reads no neighbours and no old value.
// Launch: sweep_grid(d), block SOR_THREADS.
template <bool FIRST, bool FLAT>
__global__ void __launch_bounds__(SOR_THREADS)
sor_sweep_kernel(PDims d, int colour, float omega, float h2, SorDiag dg, float *__restrict__ ec,
                 const float *__restrict__ eo, const float *__restrict__ rc)
{
    // Programmatic dependent launch: the next half-sweep may be scheduled
    // as soon as every block of this one has started, and this one reads
    // nothing before the previous grid has completed and its writes are
    // visible (both are no-ops for a launch without that dependency).
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
    int j, s0;
    if (FLAT) {
        const int ngroups = ((d.nx + 1) / 2 + 3) >> 2;
        const int t = blockIdx.x * SOR_THREADS + threadIdx.x;
        j = t / ngroups + 1;
        s0 = 4 * (t - (j - 1) * ngroups);
        if (j > d.ny) return;
    } else {
        s0 = 4 * (blockIdx.x * 32 + (threadIdx.x & 31));
        j = blockIdx.y * (SOR_THREADS / 32) + (threadIdx.x >> 5) + 1;
        if (2 * s0 + 1 > d.nx || j > d.ny) return;  // no cell of either colour in this group
    }
    const int jm = (j == 1) ? d.ny : j - 1;
    const int jp = (j == d.ny) ? 1 : j + 1;
    const bool need_nb = !FIRST || colour == 1;  // on the first red half-sweep every neighbour is still 0
    const int o = j * d.cpitch + SOR_SLOT0 + s0;  // offset inside a colour plane
    const int oym = o + (jm - j) * d.cpitch, oyp = o + (jp - j) * d.cpitch;
    const int cpl = (int)d.cplane;
#if GBSW_DEBUG_BOUNDS
    const long long nc = (long long)d.cplane * (d.nz + 2);  // elements of each colour array
#endif
#define SOR_OK4(idx) GBSW_INBOUNDS((long long)(idx), nc - 3, &g_sor_bounds)
#define SOR_OK1(idx) GBSW_INBOUNDS((long long)(idx), nc, &g_sor_bounds)
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int h = 0; h < SOR_KZ; ++h) {
        const int k = SOR_KZ * blockIdx.z + 1 + h;
        if (k > d.nz) break;
        const int q = (colour + 1 + j + k) & 1;
        const size_t plane = (size_t)k * d.cplane;
        float *__restrict__ ep = ec + plane;
        const float *__restrict__ op = eo + plane;
        // diagonal of this plane inside a row (index 1), at i = 1 (0) and at i = nx (2)
        const bool mid = k != 1 && k != d.nz;
        const float d_in = mid ? dg.d[2] : dg.d[1], y_in = mid ? dg.y[2] : dg.y[1];
        const float d_lo = mid ? dg.d[1] : dg.d[0], y_lo = mid ? dg.y[1] : dg.y[0];
        const float d_hi = mid ? dg.d[3] : dg.d[2], y_hi = mid ? dg.y[3] : dg.y[2];
        const float4 e_old = (FIRST || !SOR_OK4(plane + o)) ? zero4 : *reinterpret_cast<const float4 *>(ep + o);
        const float4 r4 = SOR_OK4(plane + o) ? *reinterpret_cast<const float4 *>(rc + plane + o) : zero4;
        float sx[4] = {0.f, 0.f, 0.f, 0.f}, sy[4] = {0.f, 0.f, 0.f, 0.f}, sz[4] = {0.f, 0.f, 0.f, 0.f};
        if (need_nb) {
            const float4 oc = SOR_OK4(plane + o) ? *reinterpret_cast<const float4 *>(op + o) : zero4;
            const float4 zm = SOR_OK4(plane + o - cpl) ? *reinterpret_cast<const float4 *>(op + o - cpl) : zero4;
            const float4 zp = SOR_OK4(plane + o + cpl) ? *reinterpret_cast<const float4 *>(op + o + cpl) : zero4;
            const float4 ym = SOR_OK4(plane + oym) ? *reinterpret_cast<const float4 *>(op + oym) : zero4;
            const float4 yp = SOR_OK4(plane + oyp) ? *reinterpret_cast<const float4 *>(op + oyp) : zero4;
            // x neighbours of slot s are slots s - 1 + q and s + q of the other colour
            if (FLAT) {
                const float xe = SOR_OK1(plane + o + (q ? 4 : -1)) ? op[o + (q ? 4 : -1)] : 0.0f;
                const float w[6] = {xe, oc.x, oc.y, oc.z, oc.w, xe};
#pragma unroll
                for (int u = 0; u < 4; ++u) sx[u] = q ? w[u + 1] + w[u + 2] : w[u] + w[u + 1];
            } else if (q == 0) {
                const float ol = SOR_OK1(plane + o - 1) ? op[o - 1] : 0.0f;
                sx[0] = ol + oc.x; sx[1] = oc.x + oc.y; sx[2] = oc.y + oc.z; sx[3] = oc.z + oc.w;
            } else {
                const float orr = SOR_OK1(plane + o + 4) ? op[o + 4] : 0.0f;
                sx[0] = oc.x + oc.y; sx[1] = oc.y + oc.z; sx[2] = oc.z + oc.w; sx[3] = oc.w + orr;
            }
            sy[0] = ym.x + yp.x; sy[1] = ym.y + yp.y; sy[2] = ym.z + yp.z; sy[3] = ym.w + yp.w;
            sz[0] = zm.x + zp.x; sz[1] = zm.y + zp.y; sz[2] = zm.z + zp.z; sz[3] = zm.w + zp.w;
        }
        const float eo4[4] = {e_old.x, e_old.y, e_old.z, e_old.w};
        const float rr4[4] = {r4.x, r4.y, r4.z, r4.w};
        float u[4];
#pragma unroll
        for (int tt = 0; tt < 4; ++tt) {
            const int i = 2 * (s0 + tt) + 1 + q;
            const float s = need_nb ? (sx[tt] + sy[tt]) + sz[tt] : 0.0f;
            const float dc = i == 1 ? d_lo : (i == d.nx ? d_hi : d_in);
            const float yc = i == 1 ? y_lo : (i == d.nx ? y_hi : y_in);
            u[tt] = i <= d.nx ? eo4[tt] + omega * (sor_div(s - h2 * rr4[tt], dc, yc) - eo4[tt]) : 0.0f;
        }
        if (SOR_OK4(plane + o)) *reinterpret_cast<float4 *>(ep + o) = make_float4(u[0], u[1], u[2], u[3]);
    }
#undef SOR_OK4
#undef SOR_OK1
}

// r = b - A p_hi in FP64 (the correction has been folded into p_hi; r is
// stored as FP32 in the colour arrays), with block partial sums of ||r||^2
// and, with WITH_BB (once per solve), of ||b||^2.  Block (bx, j, bz): 256
// cells of row j from i = 256 bx + 1, planes POI_RES_PLANES bz + 1 ..
// (no index division).  A p_hi = (sum of neighbours - d_c p) / dx^2 with
// d_c = 6 - [i == 1] - [k == 1] - [k == nz] + [i == nx]: five FP64
// additions and one FMA per cell.  The kernel is bound by the FP64 pipe,
// so 1/dx^2 comes from the host and d_c from integer selects.
// Stencil cache (fixed-count solves): with s_out, the stencil part
// s = sum of neighbours - d_c p of every cell is also stored (padded FP64
// layout); with s_in and *s_ok != 0 (p_hi unchanged since it was stored)
// s is read instead of formed, the same value, so r is bitwise the same.
template <bool WITH_BB>
__global__ void __launch_bounds__(POI_RED_THREADS)
poisson_resid_kernel(PDims d, const float *__restrict__ b, const double *__restrict__ p_hi, float *__restrict__ r0,
                     float *__restrict__ r1, double *__restrict__ partials, const double *__restrict__ s_in,
                     const int *__restrict__ s_ok, double *__restrict__ s_out)
{
    __shared__ double red[POI_RED_THREADS / 32];
    const double r2 = d.rdx2;
    const int i = blockIdx.x * POI_RED_THREADS + threadIdx.x + 1;
    const int j = blockIdx.y + 1;
    const int jm = (j == 1) ? d.ny : j - 1;
    const int jp = (j == d.ny) ? 1 : j + 1;
    double rr = 0.0, bb = 0.0;
    const bool cached = s_in != nullptr && *s_ok != 0;
    if (i <= d.nx) {
        // cells outside the grid in x or z read as 0 (ghost values unused)
        auto P = [&](int ii, int jj, int kk) -> double {
            if (ii < 1 || ii > d.nx || kk < 1 || kk > d.nz) return 0.0;
            return p_hi[pidx(d, ii, jj, kk)];
        };
        for (int kk = 0; kk < POI_RES_PLANES; ++kk) {
            const int k = blockIdx.z * POI_RES_PLANES + kk + 1;
            if (k > d.nz) break;
            double s;
            if (cached) {
                s = s_in[pidx(d, i, j, k)];
            } else {
                const double pc = p_hi[pidx(d, i, j, k)];
                const double nb = (P(i - 1, j, k) + P(i + 1, j, k)) + (P(i, jm, k) + P(i, jp, k)) +
                                  (P(i, j, k - 1) + P(i, j, k + 1));
                // d_c = 6 - [i == 1] - [k == 1] - [k == nz] + [i == nx] in {4, .., 7}
                // (nx, nz >= 2), picked by integer selects: no FP64 operation
                const int dci = 6 - (i == 1) - (k == 1) - (k == d.nz) + (i == d.nx);
                const double dc = dci == 6 ? 6.0 : (dci == 5 ? 5.0 : (dci == 7 ? 7.0 : 4.0));
                s = fma(-dc, pc, nb);
                if (s_out) s_out[pidx(d, i, j, k)] = s;
            }
            const double bc = (double)b[pidx(d, i, j, k)];
            const double res = fma(-s, r2, bc);
            float *ra = ((i + j + k) & 1) ? r1 : r0;
            ra[cidx(d, i, j, k)] = (float)res;
            rr = fma(res, res, rr);
            if (WITH_BB) bb = fma(bc, bc, bb);
        }
    }
    rr = block_sum_f64<POI_RED_THREADS / 32>(rr, red);
    if (WITH_BB) bb = block_sum_f64<POI_RED_THREADS / 32>(bb, red);
    if (threadIdx.x == 0) {
        const int blk = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partials[2 * blk] = rr;
        if (WITH_BB) partials[2 * blk + 1] = bb;
    }
}

// Folds the partials (fixed order), updates the control block and sets the
// while-node condition: continue while rho > tol and iters < max_iter.
// The ||b||^2 partials are those of the solve's first residual.
// m: the check interval; counting: m iterations ran since the previous
// check (ctl->since of them with predict), added to iters.  predict: the
// next check is placed (see set_predicted_checks): with rho falling by the
// factor g per iteration between the last two checks, the tolerance is
// n = log(tol / rho) / log(g) iterations away, and the next check comes
// after ceil(1.03 n) + 1 of them (an iteration costs far less than a
// check, so the margin errs late), at most m and max_iter - iters.
template <bool GRAPH>
__global__ void __launch_bounds__(POI_RED_THREADS)
poisson_test_kernel(const double *__restrict__ partials, int nblocks, PoissonCtl *ctl, double tol, int max_iter,
                    int m, int counting, int predict, cudaGraphConditionalHandle handle)
{
    __shared__ double red[POI_RED_THREADS / 32];
    double rr = 0.0, bb = 0.0;
    for (int q = threadIdx.x; q < nblocks; q += blockDim.x) {
        rr += partials[2 * q];
        bb += partials[2 * q + 1];
    }
    rr = block_sum_f64<POI_RED_THREADS / 32>(rr, red);
    bb = block_sum_f64<POI_RED_THREADS / 32>(bb, red);
    if (threadIdx.x == 0) {
        if (counting) {
            ctl->iters += predict ? ctl->since : m;
        } else {
            ctl->iters = 0;
            ctl->status = DEV_OK;
        }
        ctl->rr = rr;
        ctl->bb = bb;
        const double rho = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        ctl->rho = rho;
        const bool bad = !isfinite(rr) || !isfinite(bb) || !isfinite(rho);  // a NaN b must not look converged
        if (bad) ctl->status = DEV_NONFINITE;
        const bool done = bad || bb < 1e-60 || rho <= tol || ctl->iters >= max_iter;
        ctl->done = done ? 1 : 0;
        int next = m;
        if (predict && counting && !done && rho > 0.0 && rho < ctl->rho_prev && ctl->iters > ctl->iters_prev) {
            const double lg = log(rho / ctl->rho_prev) / (double)(ctl->iters - ctl->iters_prev);  // < 0
            const double n = log(tol / rho) / lg;                                                // > 0
            if (n < (double)m) next = max(1, (int)ceil(1.03 * n) + 1);
        }
        ctl->next = max(1, min(next, max_iter - ctl->iters));
        ctl->since = 0;
        ctl->rho_prev = rho;
        ctl->iters_prev = ctl->iters;
        if (GRAPH) cudaGraphSetConditional(handle, done ? 0u : 1u);
    }
}

// Predicted checks, after each chunk of c iterations of the loop body:
// counts them and sets the condition of the check node (a check is due
// once the iterations since the last one reach ctl->next, or max_iter).
__global__ void poisson_due_kernel(PoissonCtl *ctl, int c, int max_iter, cudaGraphConditionalHandle check)
{
    if (threadIdx.x != 0) return;
    const int since = ctl->since + c;
    ctl->since = since;
    const bool due = since >= ctl->next || ctl->iters + since >= max_iter;
    cudaGraphSetConditional(check, due ? 1u : 0u);
}

// Predicted checks, end of the loop body: continue unless the last check
// found the solve done.
__global__ void poisson_continue_kernel(const PoissonCtl *ctl, cudaGraphConditionalHandle loop)
{
    if (threadIdx.x == 0) cudaGraphSetConditional(loop, ctl->done ? 0u : 1u);
}

// p_hi += e, e = 0 on the interior cells of one colour (before each check).
// Launch: grid (ceil(((nx+1)/2) / 128), ny, nz), block 128 (one-dimensional).
__global__ void poisson_fold_kernel(PDims d, int colour, double *__restrict__ p_hi, float *__restrict__ ec)
{
    const int slot = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y + 1, k = blockIdx.z + 1;
    const int i = 2 * slot + 1 + ((colour + 1 + j + k) & 1);
    if (i > d.nx) return;
    const long long c = (long long)k * d.cplane + (long long)j * d.cpitch + SOR_SLOT0 + slot;
    p_hi[pidx(d, i, j, k)] += (double)ec[c];
    ec[c] = 0.0f;
}

// Dense (nz, ny, nx) <-> padded layout copies for the standalone solve.
__global__ void poisson_scatter_kernel(PDims d, const float *__restrict__ src, float *__restrict__ dst_f,
                                       double *__restrict__ dst_d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= d.nx) return;
    const float v = src[((long long)k * d.ny + j) * d.nx + i];
    const long long c = pidx(d, i + 1, j + 1, k + 1);
    if (dst_f) dst_f[c] = v;
    if (dst_d) dst_d[c] = (double)v;
}

__global__ void poisson_gather_kernel(PDims d, const double *__restrict__ src, float *__restrict__ dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y, k = blockIdx.z;
    if (i >= d.nx) return;
    dst[((long long)k * d.ny + j) * d.nx + i] = (float)src[pidx(d, i + 1, j + 1, k + 1)];
}

// ---------------------------------------------------------------------------

// Launch shape of sor_sweep_kernel: the warp-per-row mapping when a row
// holds a whole number of 32-group warps, else the flat one.
static bool sweep_flat(const PDims &d)
{
    return ((((d.nx + 1) / 2) + 3) / 4) % 32 != 0;
}

static dim3 sweep_grid(const PDims &d)
{
    const long long ngroups = (((d.nx + 1) / 2) + 3) / 4;
    if (sweep_flat(d)) return dim3(ceil_div(ngroups * d.ny, SOR_THREADS), 1, ceil_div(d.nz, SOR_KZ));
    return dim3(ceil_div(ngroups, 32), ceil_div(d.ny, SOR_THREADS / 32), ceil_div(d.nz, SOR_KZ));
}

// Enqueue one colour half-sweep.  after_sweep: the previous launch on the
// stream is a half-sweep, so this one may start programmatically (its
// blocks are scheduled during the previous sweep's last wave and wait in
// griddepcontrol.wait for its completion).
template <bool FIRST>
static cudaError_t launch_sweep(const PDims &d, int colour, float om, float h2, float *ec, const float *eo,
                                const float *rc, cudaStream_t s, bool after_sweep)
{
    const SorDiag dg = sor_diag();
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = sweep_grid(d);
    cfg.blockDim = dim3(SOR_THREADS);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = after_sweep ? attr : nullptr;
    cfg.numAttrs = after_sweep ? 1 : 0;
    if (sweep_flat(d))
        return cudaLaunchKernelEx(&cfg, sor_sweep_kernel<FIRST, true>, d, colour, om, h2, dg, ec, eo, rc);
    return cudaLaunchKernelEx(&cfg, sor_sweep_kernel<FIRST, false>, d, colour, om, h2, dg, ec, eo, rc);
}

// m red-black iterations; with from_zero the first starts from e = 0
// (FIRST: its red half-sweep reads no neighbours).
static cudaError_t launch_iterations(const PDims &d, int m, float om, float h2, float *const e[2],
                                     float *const r[2], cudaStream_t s, bool from_zero = true)
{
    cudaError_t err = cudaSuccess;
    for (int it = 0; it < m && err == cudaSuccess; ++it) {
        if (it == 0 && from_zero) {
            err = launch_sweep<true>(d, 0, om, h2, e[0], e[1], r[0], s, false);
            if (err == cudaSuccess) err = launch_sweep<true>(d, 1, om, h2, e[1], e[0], r[1], s, true);
        } else {
            err = launch_sweep<false>(d, 0, om, h2, e[0], e[1], r[0], s, it > 0);
            if (err == cudaSuccess) err = launch_sweep<false>(d, 1, om, h2, e[1], e[0], r[1], s, true);
        }
    }
    return err;
}

gbsw_status PoissonSolver::init(int nx, int ny, int nz, double dx, const float *b_dev, cudaStream_t s)
{
    d.nx = nx;
    d.ny = ny;
    d.nz = nz;
    d.pitch = (int)round_up((size_t)nx + 2, 32);
    d.plane = (long long)(ny + 2) * d.pitch;
    d.cpitch = SOR_SLOT0 + (int)round_up((size_t)(nx + 1) / 2, 4) + 4;
    d.cplane = (long long)(ny + 2) * d.cpitch;
    d.dx = dx;
    d.rdx2 = 1.0 / (dx * dx);
    b = b_dev;
    stream = s;
    const size_t n = (size_t)d.plane * (size_t)(nz + 2);
    const size_t nc = (size_t)d.cplane * (size_t)(nz + 2);
    GBSW_CUDA_TRY(cudaMalloc((void **)&p_hi, n * sizeof(double)));
    GBSW_CUDA_TRY(cudaMemsetAsync(p_hi, 0, n * sizeof(double), stream));
    for (int c = 0; c < 2; ++c) {
        GBSW_CUDA_TRY(cudaMalloc((void **)&e[c], nc * sizeof(float)));
        GBSW_CUDA_TRY(cudaMalloc((void **)&r[c], nc * sizeof(float)));
        GBSW_CUDA_TRY(cudaMemsetAsync(e[c], 0, nc * sizeof(float), stream));
        GBSW_CUDA_TRY(cudaMemsetAsync(r[c], 0, nc * sizeof(float), stream));
    }
    rgrid = dim3(ceil_div(nx, POI_RED_THREADS), ny, ceil_div(nz, POI_RES_PLANES));
    rblocks = (int)(rgrid.x * rgrid.y * rgrid.z);
    GBSW_CUDA_TRY(cudaMalloc((void **)&partials, 2 * (size_t)rblocks * sizeof(double)));
    GBSW_CUDA_TRY(cudaMalloc((void **)&ctl, sizeof(PoissonCtl)));
    GBSW_CUDA_TRY(cudaMemsetAsync(ctl, 0, sizeof(PoissonCtl), stream));
    dirty_ = true;
    return GBSW_OK;
}

void PoissonSolver::release()
{
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    if (fixed_exec_) cudaGraphExecDestroy(fixed_exec_);
    exec_ = nullptr;
    graph_ = nullptr;
    fixed_exec_ = nullptr;
    cudaFree(p_hi);
    for (int c = 0; c < 2; ++c) {
        cudaFree(e[c]);
        cudaFree(r[c]);
        e[c] = r[c] = nullptr;
    }
    cudaFree(partials);
    cudaFree(ctl);
    cudaFree(s_cache);
    cudaFree(s_ok);
    s_cache = nullptr;
    s_ok = nullptr;
    s_valid_ = false;
    p_hi = nullptr;
    partials = nullptr;
    ctl = nullptr;
}

gbsw_status PoissonSolver::configure(double omega_, double tol_, int max_iter_, int check_every)
{
    if (!(omega_ > 0.0 && omega_ < 2.0) || !(tol_ >= 0.0) || max_iter_ < 0 || check_every < 1 || check_every > 1000)
        return GBSW_ERR_ARG;
    if (omega_ != omega || tol_ != tol || max_iter_ != max_iter || check_every != m) dirty_ = true;
    if (omega_ != omega) fixed_dirty_ = true;
    omega = omega_;
    tol = tol_;
    max_iter = max_iter_;
    m = check_every;
    return GBSW_OK;
}

void PoissonSolver::set_predicted_checks(bool on)
{
    if (on != predict_) dirty_ = true;
    predict_ = on;
}

gbsw_status PoissonSolver::build_graph()
{
    if (predict_) return build_graph_predicted();
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    exec_ = nullptr;
    graph_ = nullptr;

    const size_t nc = (size_t)d.cplane * (size_t)(d.nz + 2);
    const float om = (float)omega, h2 = (float)(d.dx * d.dx);
    const int nxh = (d.nx + 1) / 2;
    const dim3 fgrid(ceil_div(nxh, 128), d.ny, d.nz), fblock(128);

    cudaStream_t cs = nullptr;
    GBSW_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraphConditionalHandle handle;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t cnode;
    cudaGraph_t body;
    cudaError_t err = cudaSuccess;
    auto chk = [&](cudaError_t e2) {
        if (err == cudaSuccess && e2 != cudaSuccess) err = e2;
    };
    chk(cudaGraphCreate(&graph_, 0));
    chk(cudaGraphConditionalHandleCreate(&handle, graph_, 0, cudaGraphCondAssignDefault));
    chk(cudaStreamBeginCaptureToGraph(cs, graph_, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if (err == cudaSuccess) {
        // prelude: e = 0, r = b - A p_hi, ||b||^2, first test
        chk(cudaMemsetAsync(e[0], 0, nc * sizeof(float), cs));
        chk(cudaMemsetAsync(e[1], 0, nc * sizeof(float), cs));
        poisson_resid_kernel<true><<<rgrid, POI_RED_THREADS, 0, cs>>>(d, b, p_hi, r[0], r[1], partials, nullptr, nullptr, nullptr);
        chk(cudaGetLastError());
        poisson_test_kernel<true><<<1, POI_RED_THREADS, 0, cs>>>(partials, rblocks, ctl, tol, max_iter, m, 0,
                                                                  0, handle);
        chk(cudaGetLastError());
        // while node
        cudaStreamCaptureStatus cst;
        cudaGraph_t cap_graph;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        chk(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cap_graph, &deps, nullptr, &ndeps));
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = handle;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        if (err == cudaSuccess) chk(cudaGraphAddNode(&cnode, cap_graph, deps, nullptr, ndeps, &cp));
        if (err == cudaSuccess) chk(cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    }
    cudaGraph_t captured = nullptr;
    cudaError_t e_end = cudaStreamEndCapture(cs, &captured);
    chk(e_end);
    if (err == cudaSuccess) {
        // body of the while node: m iterations, fold, residual, test (the
        // fold leaves p_hi complete whenever the loop stops)
        body = cp.conditional.phGraph_out[0];
        chk(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        if (err == cudaSuccess) {
            chk(launch_iterations(d, m, om, h2, e, r, cs));
            poisson_fold_kernel<<<fgrid, fblock, 0, cs>>>(d, 0, p_hi, e[0]);
            poisson_fold_kernel<<<fgrid, fblock, 0, cs>>>(d, 1, p_hi, e[1]);
            poisson_resid_kernel<false><<<rgrid, POI_RED_THREADS, 0, cs>>>(d, b, p_hi, r[0], r[1], partials, nullptr, nullptr, nullptr);
            poisson_test_kernel<true><<<1, POI_RED_THREADS, 0, cs>>>(partials, rblocks, ctl, tol, max_iter, m,
                                                                    1, 0, handle);
            chk(cudaGetLastError());
        }
        cudaGraph_t body_out = nullptr;
        chk(cudaStreamEndCapture(cs, &body_out));
    }
    if (err == cudaSuccess) chk(cudaGraphInstantiate(&exec_, graph_, 0));
    cudaStreamDestroy(cs);
    if (err != cudaSuccess) {
        record_cuda_error(err, "poisson graph build", __FILE__, __LINE__);
        return GBSW_ERR_CUDA;
    }
    dirty_ = false;
    return GBSW_OK;
}

// The solve graph with predicted checks: prelude (e = 0, first residual,
// test), then a while node whose body is a chunk of c iterations (c the
// largest divisor of m up to SOR_CHUNK_MAX, or SOR_CHUNK_MAX when that
// divisor is small), poisson_due_kernel, an if
// node holding the check (fold, FP64 residual, test with prediction) and
// poisson_continue_kernel.  Every chunk starts from the correction as the
// last chunk or check left it; after a check it is 0, where the general
// red half-sweep gives bitwise what the FIRST one does.
gbsw_status PoissonSolver::build_graph_predicted()
{
    if (exec_) cudaGraphExecDestroy(exec_);
    if (graph_) cudaGraphDestroy(graph_);
    exec_ = nullptr;
    graph_ = nullptr;

    int c = 1;
    for (int x = std::min(m, SOR_CHUNK_MAX); x >= 1; --x)
        if (m % x == 0) {
            c = x;
            break;
        }
    // An interval with no divisor near SOR_CHUNK_MAX (a prime above it, say)
    // would give chunks of a few iterations, each paying two control
    // kernels: take full chunks, and the check then comes at the first
    // chunk boundary at or past the interval.
    if (c < SOR_CHUNK_MAX / 4 && m > SOR_CHUNK_MAX) c = SOR_CHUNK_MAX;
    const size_t nc = (size_t)d.cplane * (size_t)(d.nz + 2);
    const float om = (float)omega, h2 = (float)(d.dx * d.dx);
    const int nxh = (d.nx + 1) / 2;
    const dim3 fgrid(ceil_div(nxh, 128), d.ny, d.nz), fblock(128);

    cudaStream_t cs = nullptr;
    GBSW_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t err = cudaSuccess;
    auto chk = [&](cudaError_t e2) {
        if (err == cudaSuccess && e2 != cudaSuccess) err = e2;
    };
    // Add a conditional node of the given type at the current capture
    // point of cs and make it the capture's only dependency; its body graph
    // goes to *body.
    auto add_conditional = [&](cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, cudaGraph_t *body) {
        cudaStreamCaptureStatus cst;
        cudaGraph_t cap_graph;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        chk(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cap_graph, &deps, nullptr, &ndeps));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = type;
        cp.conditional.size = 1;
        cudaGraphNode_t node;
        if (err == cudaSuccess) chk(cudaGraphAddNode(&node, cap_graph, deps, nullptr, ndeps, &cp));
        if (err == cudaSuccess)
            chk(cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        *body = err == cudaSuccess ? cp.conditional.phGraph_out[0] : nullptr;
    };
    cudaGraphConditionalHandle hloop = 0, hcheck = 0;
    cudaGraph_t body = nullptr, check_body = nullptr;
    chk(cudaGraphCreate(&graph_, 0));
    chk(cudaGraphConditionalHandleCreate(&hloop, graph_, 0, cudaGraphCondAssignDefault));
    chk(cudaStreamBeginCaptureToGraph(cs, graph_, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    if (err == cudaSuccess) {
        // prelude: e = 0, r = b - A p_hi, ||b||^2, first test (next = m)
        chk(cudaMemsetAsync(e[0], 0, nc * sizeof(float), cs));
        chk(cudaMemsetAsync(e[1], 0, nc * sizeof(float), cs));
        poisson_resid_kernel<true><<<rgrid, POI_RED_THREADS, 0, cs>>>(d, b, p_hi, r[0], r[1], partials, nullptr, nullptr, nullptr);
        chk(cudaGetLastError());
        poisson_test_kernel<true><<<1, POI_RED_THREADS, 0, cs>>>(partials, rblocks, ctl, tol, max_iter, m, 0, 1,
                                                                  hloop);
        chk(cudaGetLastError());
        add_conditional(hloop, cudaGraphCondTypeWhile, &body);
    }
    cudaGraph_t captured = nullptr;
    chk(cudaStreamEndCapture(cs, &captured));
    if (err == cudaSuccess) {
        // loop body: c iterations, due test, check node, loop condition
        chk(cudaGraphConditionalHandleCreate(&hcheck, body, 0, cudaGraphCondAssignDefault));
        chk(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        if (err == cudaSuccess) {
            chk(launch_iterations(d, c, om, h2, e, r, cs, false));
            poisson_due_kernel<<<1, 32, 0, cs>>>(ctl, c, max_iter, hcheck);
            chk(cudaGetLastError());
            add_conditional(hcheck, cudaGraphCondTypeIf, &check_body);
            poisson_continue_kernel<<<1, 32, 0, cs>>>(ctl, hloop);
            chk(cudaGetLastError());
        }
        cudaGraph_t body_out = nullptr;
        chk(cudaStreamEndCapture(cs, &body_out));
    }
    if (err == cudaSuccess) {
        // check: fold the correction into p_hi, FP64 residual, test and prediction
        chk(cudaStreamBeginCaptureToGraph(cs, check_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        if (err == cudaSuccess) {
            poisson_fold_kernel<<<fgrid, fblock, 0, cs>>>(d, 0, p_hi, e[0]);
            poisson_fold_kernel<<<fgrid, fblock, 0, cs>>>(d, 1, p_hi, e[1]);
            poisson_resid_kernel<false><<<rgrid, POI_RED_THREADS, 0, cs>>>(d, b, p_hi, r[0], r[1], partials, nullptr, nullptr, nullptr);
            poisson_test_kernel<false><<<1, POI_RED_THREADS, 0, cs>>>(partials, rblocks, ctl, tol, max_iter, m, 1,
                                                                     1, 0);
            chk(cudaGetLastError());
        }
        cudaGraph_t check_out = nullptr;
        chk(cudaStreamEndCapture(cs, &check_out));
    }
    if (err == cudaSuccess) chk(cudaGraphInstantiate(&exec_, graph_, 0));
    cudaStreamDestroy(cs);
    if (err != cudaSuccess) {
        record_cuda_error(err, "poisson graph build (predicted checks)", __FILE__, __LINE__);
        return GBSW_ERR_CUDA;
    }
    dirty_ = false;
    return GBSW_OK;
}

gbsw_status PoissonSolver::enqueue()
{
    s_valid_ = false;  // the folds change p_hi and no stencil is stored
    if (dirty_) {
        gbsw_status st = build_graph();
        if (st != GBSW_OK) return st;
    }
    GBSW_CUDA_TRY(cudaGraphLaunch(exec_, stream));
    return GBSW_OK;
}

gbsw_status PoissonSolver::enqueue_fixed(int niter, bool use_graph)
{
    if (niter < 0) return GBSW_ERR_ARG;
    if (!s_cache) {  // the stencil cache (allocated once: the captured graph holds its address)
        const size_t n = (size_t)d.plane * (size_t)(d.nz + 2);
        GBSW_CUDA_TRY(cudaMalloc((void **)&s_cache, n * sizeof(double)));
        GBSW_CUDA_TRY(cudaMalloc((void **)&s_ok, sizeof(int)));
        s_valid_ = false;
    }
    // the first residual may reuse the last fixed-count solve's stencil only
    // if p_hi has not changed since
    GBSW_CUDA_TRY(cudaMemsetAsync(s_ok, s_valid_ ? 1 : 0, sizeof(int), stream));
    s_valid_ = false;  // set again once this solve, whose final residual stores the stencil, is enqueued
    if (!use_graph || niter > SOR_FIXED_GRAPH_MAX_ITER) {
        const gbsw_status st = record_fixed(niter, stream);
        s_valid_ = st == GBSW_OK;
        return st;
    }
    if (!fixed_exec_ || fixed_niter_ != niter || fixed_dirty_) {
        if (fixed_exec_) cudaGraphExecDestroy(fixed_exec_);
        fixed_exec_ = nullptr;
        cudaStream_t cs = nullptr;
        GBSW_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        gbsw_status st = GBSW_OK;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = record_fixed(niter, cs);
            e = cudaStreamEndCapture(cs, &g);
        }
        if (e == cudaSuccess && st == GBSW_OK) e = cudaGraphInstantiate(&fixed_exec_, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess || st != GBSW_OK) {
            if (e != cudaSuccess) record_cuda_error(e, "poisson fixed-count graph", __FILE__, __LINE__);
            fixed_exec_ = nullptr;
            return st != GBSW_OK ? st : GBSW_ERR_CUDA;
        }
        fixed_niter_ = niter;
        fixed_dirty_ = false;
    }
    GBSW_CUDA_TRY(cudaGraphLaunch(fixed_exec_, stream));
    s_valid_ = true;
    return GBSW_OK;
}

gbsw_status PoissonSolver::record_fixed(int niter, cudaStream_t stream)
{
    const size_t nc = (size_t)d.cplane * (size_t)(d.nz + 2);
    const float om = (float)omega, h2 = (float)(d.dx * d.dx);
    const dim3 fgrid(ceil_div((d.nx + 1) / 2, 128), d.ny, d.nz), fblock(128);
    GBSW_CUDA_TRY(cudaMemsetAsync(e[0], 0, nc * sizeof(float), stream));
    GBSW_CUDA_TRY(cudaMemsetAsync(e[1], 0, nc * sizeof(float), stream));
    poisson_resid_kernel<true><<<rgrid, POI_RED_THREADS, 0, stream>>>(d, b, p_hi, r[0], r[1], partials, s_cache, s_ok,
                                                                      nullptr);
    poisson_test_kernel<false><<<1, POI_RED_THREADS, 0, stream>>>(partials, rblocks, ctl, 0.0, niter, 0, 0, 0, 0);
    cudaError_t err = launch_iterations(d, niter, om, h2, e, r, stream);
    if (err != cudaSuccess) {
        record_cuda_error(err, "SOR sweep launch", __FILE__, __LINE__);
        return GBSW_ERR_CUDA;
    }
    poisson_fold_kernel<<<fgrid, fblock, 0, stream>>>(d, 0, p_hi, e[0]);
    poisson_fold_kernel<<<fgrid, fblock, 0, stream>>>(d, 1, p_hi, e[1]);
    poisson_resid_kernel<false><<<rgrid, POI_RED_THREADS, 0, stream>>>(d, b, p_hi, r[0], r[1], partials, nullptr,
                                                                       nullptr, s_cache);
    poisson_test_kernel<false><<<1, POI_RED_THREADS, 0, stream>>>(partials, rblocks, ctl, 0.0, niter, niter,
                                                                   1, 0, 0);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status PoissonSolver::record(PoissonCtl *dst)
{
    GBSW_CUDA_TRY(cudaMemcpyAsync(dst, ctl, sizeof(PoissonCtl), cudaMemcpyDeviceToDevice, stream));
    return GBSW_OK;
}

}  // namespace gbsw

using namespace gbsw;

extern "C" gbsw_status poisson_solve(int nx, int ny, int nz, double dx, float *p, const float *b, double omega,
                                     double tol, int max_iter, int check_every, void *stream, int *iters,
                                     double *rel_res)
{
    gbsw::NvtxRange nvtx_range("poisson_solve");
    if (nx < 2 || ny < 2 || nz < 2 || (ny & 1) || nx > 8192 || ny > 8192 || nz > 8192 || !(dx > 0) || !p || !b)
        return GBSW_ERR_ARG;
    const bool fixed = tol < 0.0;  // paper mode: exactly max_iter iterations, no convergence test
    cudaStream_t s = (cudaStream_t)stream;
    PoissonSolver S;
    float *bp = nullptr;
    gbsw_status st = GBSW_OK;
    PoissonCtl host{};
    do {
        PDims d0;
        d0.pitch = (int)round_up((size_t)nx + 2, 32);
        d0.plane = (long long)(ny + 2) * d0.pitch;
        const size_t np = (size_t)d0.plane * (size_t)(nz + 2);
        cudaError_t e = cudaMalloc((void **)&bp, np * sizeof(float));
        if (e != cudaSuccess) {
            record_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
            st = GBSW_ERR_OOM;
            break;
        }
        if ((e = cudaMemsetAsync(bp, 0, np * sizeof(float), s)) != cudaSuccess) {
            st = GBSW_ERR_CUDA;
            break;
        }
        st = S.init(nx, ny, nz, dx, bp, s);
        if (st != GBSW_OK) break;
        st = S.configure(omega, fixed ? 0.0 : tol, max_iter, check_every);
        if (st != GBSW_OK) break;
        const dim3 g(ceil_div(nx, 128), ny, nz), blk(128);
        poisson_scatter_kernel<<<g, blk, 0, s>>>(S.d, b, bp, nullptr);
        poisson_scatter_kernel<<<g, blk, 0, s>>>(S.d, p, nullptr, S.p_hi);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            record_cuda_error(e, "poisson scatter", __FILE__, __LINE__);
            st = GBSW_ERR_CUDA;
            break;
        }
        st = fixed ? S.enqueue_fixed(max_iter, false) : S.enqueue();
        if (st != GBSW_OK) break;
        poisson_gather_kernel<<<g, blk, 0, s>>>(S.d, S.p_hi, p);
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(&host, S.ctl, sizeof(PoissonCtl), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            record_cuda_error(e, "poisson solve", __FILE__, __LINE__);
            st = GBSW_ERR_CUDA;
            break;
        }
    } while (0);
    S.release();
    cudaFree(bp);
    if (st != GBSW_OK) return st;
    if (iters) *iters = host.iters;
    if (rel_res) *rel_res = host.rho;
    if (host.status != DEV_OK) return dev_status_to_gbsw(host.status);
    if (fixed) return GBSW_OK;
    return host.done && (host.rho <= tol || host.bb < 1e-60) ? GBSW_OK : GBSW_NOT_CONVERGED;
}

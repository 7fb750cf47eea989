// 2-D shallow-water time step (Sec. 6.2 of arXiv:1711.04471: the predictor
// "dyn", the first-order Shapiro filter "shapiro" and the state update),
// as one fused, temporally blocked CUDA kernel, plus the FP64 volume
// reduction.  The three map kernels the paper's compiler generates for this
// loop are fused into one streaming kernel (sw_stream.cuh) that reads the
// state once and writes it once per T time steps.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "sw_kernels.cuh"
#include "sw_stream.cuh"
#include "sw_tile.cuh"

using namespace gbsw;

namespace gbsw {

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

struct gbsw_sw {
    gbsw_sw_params p;
    SWDev d;
    cudaStream_t stream;
    float *H;
    float *eta[2], *u[2], *v[2];
    int cur;
    int blocking;           // 0 = automatic
    int rows;               // row-segment height of a CTA, 0 = automatic
    // CUDA graphs of SW_CHUNK fused launches of depth chunk_T starting from
    // buffer set 0 or 1, replayed by sw_step (rebuilt when the tiling changes)
    cudaGraphExec_t chunk[2];
    int chunk_T, chunk_rows;
    double *partials;       // SW_VOL_BLOCKS * 3 doubles (scratch of the volume reduction)
    double *result;         // 3 doubles on the device
    double *h_result;       // 3 doubles, pinned host
    uint8_t *wet;           // ny*nx bytes, staging for sw_get_state
};

namespace {

constexpr int SW_CHUNK = 32;  // fused launches per replayed graph (even: a chunk ends on its start buffer)

// Resident CTAs per SM of the depth-T streaming kernel.
template <int T>
int stream_per_sm()
{
    static int per_sm = 0;
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sw_stream_kernel<T>, SWS_THREADS, 0) !=
            cudaSuccess)
            per_sm = 0;
        if (per_sm < 1) per_sm = 1;
    }
    return per_sm;
}

int stream_per_sm(int T)
{
    switch (T) {
    case 1: return stream_per_sm<1>();
    case 2: return stream_per_sm<2>();
    case 3: return stream_per_sm<3>();
    case 4: return stream_per_sm<4>();
    case 5: return stream_per_sm<5>();
    default: return stream_per_sm<6>();
    }
}

// Default row-segment height: one wave of CTAs sized from the occupancy,
// every resident CTA one (strip, row segment), with segments kept well
// above the pipeline depth (3T - 1 rows of fill per segment).
int default_rows(const gbsw_sw *s, int T)
{
    const int strips = ceil_div(s->d.nx, SWS_THREADS - 4 * T);
    const int capacity = stream_per_sm(T) * sm_count();
    int segments = std::max(1, capacity / strips);
    segments = std::min(segments, std::max(1, s->d.ny / (8 * T)));
    return ceil_div(s->d.ny, segments);
}

// Streaming launch of depth T over row segments of `rows` rows.
template <int T>
cudaError_t launch_stream(const gbsw_sw *s, int rows, cudaStream_t st, const float *eta_in, const float *u_in,
                          const float *v_in, float *eta_out, float *u_out, float *v_out)
{
    constexpr int W = SWS_THREADS - 4 * T;
    const int strips = ceil_div(s->d.nx, W);
    const int segments = ceil_div(s->d.ny, rows);
    dim3 grid(strips, segments);
    sw_stream_kernel<T><<<grid, SWS_THREADS, 0, st>>>(s->d, rows, s->H, eta_in, u_in, v_in, eta_out, u_out, v_out);
    return cudaGetLastError();
}

// Written rows of a tile for the tiling code rows < 0: -1 the default
// height, -h (h >= 2) h rows.
int tile_rows(int rows) { return rows == -1 ? SWT_H : -rows; }

// Resident CTAs per SM of the depth-T tile kernel.
template <int T>
int tile_per_sm()
{
    static int per_sm = 0;
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sw_tile_kernel<T>, SWT_THREADS, 0) !=
            cudaSuccess)
            per_sm = 0;
        if (per_sm < 1) per_sm = 1;
    }
    return per_sm;
}

int tile_per_sm(int T)
{
    switch (T) {
    case 1: return tile_per_sm<1>();
    case 2: return tile_per_sm<2>();
    default: return tile_per_sm<3>();
    }
}

// Tile height that spreads a tile launch most evenly over the resident
// CTA slots: with c column tiles and S slots, h rows per tile take
// ceil(c ceil(ny / h) / S) rounds of CTAs, each about as long as one
// tile's (SWT_W + 4T)(h + 4T) cells of work; the least rounds x (h + 4T)
// wins (ties: the taller tile).  Heights below 8 rows are not considered.
int balanced_tile_rows(const gbsw_sw *s, int T)
{
    const long long c = ceil_div(s->d.nx, SWT_W);
    const long long slots = (long long)tile_per_sm(T) * sm_count();
    int best = SWT_H;
    long long best_cost = -1;
    for (int h = swt_max_rows(T); h >= 8; --h) {
        const long long rounds = (c * ceil_div(s->d.ny, h) + slots - 1) / slots;
        const long long cost = rounds * (h + 4 * T);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = h;
        }
    }
    return best;
}

// One launch of the tile kernel of depth T (1..SWT_MAX_T) with th written
// rows per tile.  after_tile: the previous launch on the stream is a tile
// launch, so this one may start programmatically (its blocks are scheduled
// while the previous launch drains and wait in griddepcontrol.wait for its
// completion).
template <int T>
cudaError_t launch_tile(const gbsw_sw *s, int th, cudaStream_t st, const float *eta_in, const float *u_in,
                        const float *v_in, float *eta_out, float *u_out, float *v_out, bool after_tile)
{
    if (th < 2 || th > swt_max_rows(T)) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ceil_div(s->d.nx, SWT_W), ceil_div(s->d.ny, th));
    cfg.blockDim = dim3(SWT_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = after_tile ? attr : nullptr;
    cfg.numAttrs = after_tile ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, sw_tile_kernel<T>, s->d, th, (const float *)s->H, eta_in, u_in, v_in, eta_out,
                              u_out, v_out);
}

// One launch of depth T from buffer set a into the other one, on stream st:
// rows > 0 the streaming kernel over row segments of that height, rows < 0
// the tile kernel with tile_rows(rows) rows per tile.  after_tile (tile
// launches only): the previous launch on the stream is a tile launch.
cudaError_t launch_from(const gbsw_sw *s, int T, int rows, int a, cudaStream_t st, bool after_tile = false)
{
    const int b = 1 - a;
    const float *ei = s->eta[a], *ui = s->u[a], *vi = s->v[a];
    float *eo = s->eta[b], *uo = s->u[b], *vo = s->v[b];
    if (rows < 0) {
        switch (T) {
        case 1: return launch_tile<1>(s, tile_rows(rows), st, ei, ui, vi, eo, uo, vo, after_tile);
        case 2: return launch_tile<2>(s, tile_rows(rows), st, ei, ui, vi, eo, uo, vo, after_tile);
        case 3: return launch_tile<3>(s, tile_rows(rows), st, ei, ui, vi, eo, uo, vo, after_tile);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (T) {
    case 1: return launch_stream<1>(s, rows, st, ei, ui, vi, eo, uo, vo);
    case 2: return launch_stream<2>(s, rows, st, ei, ui, vi, eo, uo, vo);
    case 3: return launch_stream<3>(s, rows, st, ei, ui, vi, eo, uo, vo);
    case 4: return launch_stream<4>(s, rows, st, ei, ui, vi, eo, uo, vo);
    case 5: return launch_stream<5>(s, rows, st, ei, ui, vi, eo, uo, vo);
    case 6: return launch_stream<6>(s, rows, st, ei, ui, vi, eo, uo, vo);
    default: return cudaErrorInvalidValue;
    }
}

int auto_blocking(const gbsw_sw *) { return 3; }

int tiling_T(const gbsw_sw *s) { return s->blocking > 0 ? s->blocking : auto_blocking(s); }

int tiling_rows(const gbsw_sw *s, int T) { return s->rows != 0 ? s->rows : default_rows(s, T); }

void drop_chunks(gbsw_sw *s)
{
    for (int k = 0; k < 2; ++k) {
        if (s->chunk[k]) cudaGraphExecDestroy(s->chunk[k]);
        s->chunk[k] = nullptr;
    }
}

// The graph of SW_CHUNK launches of depth T starting from buffer set a
// (captured on a private stream, replayed on the context's stream).
cudaError_t chunk_graph(gbsw_sw *s, int T, int rows, int a, cudaGraphExec_t *out)
{
    if (s->chunk_T != T || s->chunk_rows != rows) {
        drop_chunks(s);
        s->chunk_T = T;
        s->chunk_rows = rows;
    }
    if (s->chunk[a]) {
        *out = s->chunk[a];
        return cudaSuccess;
    }
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t el = cudaSuccess;
        for (int k = 0; k < SW_CHUNK && el == cudaSuccess; ++k)
            el = launch_from(s, T, rows, (a + k) & 1, cs, rows < 0 && k > 0);
        e = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = el;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->chunk[a], g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        s->chunk[a] = nullptr;
        return e;
    }
    *out = s->chunk[a];
    return cudaSuccess;
}

// nsteps time steps with depth-T launches over `rows`-row segments: whole
// chunks of SW_CHUNK launches as graph replays, the rest launched directly.
gbsw_status run_steps(gbsw_sw *s, int nsteps, int T, int rows)
{
    int full = nsteps / T;
    const int rest = nsteps % T;
    while (full >= SW_CHUNK) {
        cudaGraphExec_t ge = nullptr;
        cudaError_t e = chunk_graph(s, T, rows, s->cur, &ge);
        if (e == cudaSuccess) e = cudaGraphLaunch(ge, s->stream);
        if (e != cudaSuccess) {
            record_cuda_error(e, "sw_step graph", __FILE__, __LINE__);
            return GBSW_ERR_CUDA;
        }
        full -= SW_CHUNK;  // even: the chunk ends on the buffer set it started from
    }
    for (int k = 0; k < full + (rest > 0); ++k) {
        const int t = k < full ? T : rest;
        cudaError_t e = launch_from(s, t, (t == T || rows < 0) ? rows : default_rows(s, t), s->cur, s->stream,
                                    rows < 0 && k > 0);
        if (e != cudaSuccess) {
            record_cuda_error(e, rows < 0 ? "sw_tile_kernel" : "sw_stream_kernel", __FILE__, __LINE__);
            return GBSW_ERR_CUDA;
        }
        s->cur = 1 - s->cur;
    }
    return GBSW_OK;
}

}  // namespace

extern "C" {

gbsw_status sw_create(const gbsw_sw_params *params, const double *H, const double *eta0, void *stream,
                      gbsw_sw **out)
{
    if (!params || !H || !eta0 || !out) return GBSW_ERR_ARG;
    const gbsw_sw_params P = *params;
    if (P.nx < 2 || P.ny < 2 || P.nx > (1 << 20) || P.ny > (1 << 20)) return GBSW_ERR_ARG;
    if (!(P.dx > 0) || !(P.dy > 0) || !(P.dt > 0) || !(P.g > 0) || !(P.eps >= 0 && P.eps <= 1) ||
        !(P.hmin >= 0))
        return GBSW_ERR_ARG;
    const size_t n = (size_t)P.nx * (size_t)P.ny;
    std::vector<float> h32(n), e32(n);
    double hmax = 0.0;
    for (size_t k = 0; k < n; ++k) {
        if (!std::isfinite(H[k]) || !std::isfinite(eta0[k])) return GBSW_ERR_ARG;
        double e = eta0[k] < -H[k] ? -H[k] : eta0[k];
        hmax = std::max(hmax, H[k] + e);
        h32[k] = (float)H[k];
        e32[k] = (float)e;
    }
    const double courant = sqrt(P.g * hmax) * P.dt * sqrt(1.0 / (P.dx * P.dx) + 1.0 / (P.dy * P.dy));
    if (courant > 1.0) return GBSW_ERR_CFL;
    if (fault_injected("alloc")) return GBSW_ERR_OOM;

    gbsw_sw *s = (gbsw_sw *)calloc(1, sizeof(gbsw_sw));
    if (!s) return GBSW_ERR_OOM;
    s->p = P;
    s->stream = (cudaStream_t)stream;
    s->d.nx = P.nx;
    s->d.ny = P.ny;
    s->d.pitch = (int)round_up((size_t)P.nx, 32);
    s->d.gdt_dx = (float)(P.g * P.dt / P.dx);
    s->d.gdt_dy = (float)(P.g * P.dt / P.dy);
    s->d.dt_dx = (float)(P.dt / P.dx);
    s->d.dt_dy = (float)(P.dt / P.dy);
    s->d.q = (float)(0.25 * P.eps);
    s->d.hmin = (float)P.hmin;

    const size_t bytes = (size_t)s->d.pitch * (size_t)P.ny * sizeof(float);
    auto fail = [&](gbsw_status code) {
        sw_destroy(s);
        return code;
    };
#define SW_ALLOC(ptr, sz)                                                      \
    do {                                                                       \
        cudaError_t _e = cudaMalloc((void **)&(ptr), (sz));                    \
        if (_e != cudaSuccess) {                                               \
            record_cuda_error(_e, "cudaMalloc", __FILE__, __LINE__);           \
            return fail(GBSW_ERR_OOM);                                         \
        }                                                                      \
    } while (0)
    SW_ALLOC(s->H, bytes);
    for (int b = 0; b < 2; ++b) {
        SW_ALLOC(s->eta[b], bytes);
        SW_ALLOC(s->u[b], bytes);
        SW_ALLOC(s->v[b], bytes);
    }
    SW_ALLOC(s->partials, SW_VOL_BLOCKS * 3 * sizeof(double));
    SW_ALLOC(s->result, 3 * sizeof(double));
    SW_ALLOC(s->wet, n);
#undef SW_ALLOC
    if (cudaMallocHost((void **)&s->h_result, 3 * sizeof(double)) != cudaSuccess) return fail(GBSW_ERR_OOM);

    cudaError_t e = cudaSuccess;
    float *all[7] = {s->H, s->eta[0], s->eta[1], s->u[0], s->u[1], s->v[0], s->v[1]};
    for (float *ptr : all)
        if (e == cudaSuccess) e = cudaMemsetAsync(ptr, 0, bytes, s->stream);
    const size_t dp = (size_t)s->d.pitch * sizeof(float), hp = (size_t)P.nx * sizeof(float);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(s->H, dp, h32.data(), hp, hp, P.ny, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(s->eta[0], dp, e32.data(), hp, hp, P.ny, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        record_cuda_error(e, "sw_create upload", __FILE__, __LINE__);
        return fail(GBSW_ERR_CUDA);
    }
    *out = s;
    return GBSW_OK;
}

gbsw_status sw_set_blocking(gbsw_sw *s, int steps_per_launch)
{
    if (!s || steps_per_launch < 0 || steps_per_launch > SW_MAX_BLOCKING) return GBSW_ERR_ARG;
    s->blocking = steps_per_launch;
    s->rows = 0;
    return GBSW_OK;
}

gbsw_status sw_set_tiling(gbsw_sw *s, int steps_per_launch, int rows)
{
    if (!s || steps_per_launch < 0 || steps_per_launch > SW_MAX_BLOCKING) return GBSW_ERR_ARG;
    if (rows < 0 && (steps_per_launch < 1 || steps_per_launch > SWT_MAX_T || rows < -swt_max_rows(steps_per_launch)))
        return GBSW_ERR_ARG;
    s->blocking = steps_per_launch;
    s->rows = rows;
    return GBSW_OK;
}

gbsw_status sw_step(gbsw_sw *s, int nsteps)
{
    gbsw::NvtxRange nvtx_range("sw_step");
    if (!s || nsteps < 0) return GBSW_ERR_ARG;
    const int T = tiling_T(s);
    return run_steps(s, nsteps, T, tiling_rows(s, T));
}

gbsw_status sw_autotune(gbsw_sw *s, int trial_steps, int *T_out, int *rows_out)
{
    gbsw::NvtxRange nvtx_range("sw_autotune");
    if (!s || trial_steps < 1 || trial_steps > 100000) return GBSW_ERR_ARG;
    const size_t fb = (size_t)s->d.pitch * (size_t)s->d.ny * sizeof(float);
    float *save[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gbsw_status st = GBSW_OK;
    int bestT = tiling_T(s), best_rows = tiling_rows(s, bestT);
    float best = INFINITY;
    const int c0 = s->cur;
    do {
        bool ok = true;
        for (int k = 0; k < 3 && ok; ++k) ok = cudaMalloc((void **)&save[k], fb) == cudaSuccess;
        if (!ok) {
            st = GBSW_ERR_OOM;
            break;
        }
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
            cudaMemcpyAsync(save[0], s->eta[c0], fb, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess ||
            cudaMemcpyAsync(save[1], s->u[c0], fb, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess ||
            cudaMemcpyAsync(save[2], s->v[c0], fb, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess) {
            st = GBSW_ERR_CUDA;
            break;
        }
        for (int T = 1; T <= SW_MAX_BLOCKING && st == GBSW_OK; ++T) {
            // segment heights: the default, and those giving 1, 2, 3 waves of resident CTAs
            const int strips = ceil_div(s->d.nx, SWS_THREADS - 4 * T);
            const int capacity = stream_per_sm(T) * sm_count();
            // tile kernel (T <= SWT_MAX_T): the default tile (-1) and the height
            // that spreads its CTAs most evenly (-h)
            int cand[6] = {default_rows(s, T), 0, 0, 0, T <= SWT_MAX_T ? -1 : 0, 0};
            for (int w = 1; w <= 3; ++w)
                cand[w] = std::max(2, ceil_div(s->d.ny, std::max(1, ceil_div(w * capacity, strips))));
            if (T <= SWT_MAX_T) {
                const int h = balanced_tile_rows(s, T);
                cand[5] = h == SWT_H ? -1 : -h;
            }
            for (int c = 0; c < 6 && st == GBSW_OK; ++c) {
                if (cand[c] == 0) continue;
                bool seen = false;
                for (int q = 0; q < c; ++q) seen |= cand[q] == cand[c];
                if (seen) continue;
                const int steps = std::max(T, trial_steps / T * T);
                if ((st = run_steps(s, steps, T, cand[c])) != GBSW_OK) break;  // warm-up (and graph capture)
                cudaEventRecord(e0, s->stream);
                if ((st = run_steps(s, steps, T, cand[c])) != GBSW_OK) break;
                cudaEventRecord(e1, s->stream);
                float ms = 0.0f;
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    st = GBSW_ERR_CUDA;
                    break;
                }
                const float per = ms / steps;
                if (per < best) {
                    best = per;
                    bestT = T;
                    best_rows = cand[c];
                }
            }
        }
        // restore the state: results do not depend on the tiling, so the
        // trials leave no trace
        const int c = s->cur;
        if (cudaMemcpyAsync(s->eta[c], save[0], fb, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess ||
            cudaMemcpyAsync(s->u[c], save[1], fb, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess ||
            cudaMemcpyAsync(s->v[c], save[2], fb, cudaMemcpyDeviceToDevice, s->stream) != cudaSuccess ||
            cudaStreamSynchronize(s->stream) != cudaSuccess)
            st = GBSW_ERR_CUDA;
    } while (0);
    for (int k = 0; k < 3; ++k) cudaFree(save[k]);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != GBSW_OK) return st;
    s->blocking = bestT;
    s->rows = best_rows;
    if (T_out) *T_out = bestT;
    if (rows_out) *rows_out = best_rows;
    return GBSW_OK;
}

gbsw_status sw_volume(gbsw_sw *s, double *volume, double *wet_volume)
{
    gbsw::NvtxRange nvtx_range("sw_volume");
    if (!s) return GBSW_ERR_ARG;
    sw_volume_partial_kernel<<<SW_VOL_BLOCKS, SW_VOL_THREADS, 0, s->stream>>>(s->d, s->H, s->eta[s->cur],
                                                                             s->partials);
    GBSW_LAUNCH_CHECK();
    sw_volume_final_kernel<<<1, SW_VOL_THREADS, 0, s->stream>>>(s->partials, SW_VOL_BLOCKS,
                                                               s->p.dx * s->p.dy, s->result);
    GBSW_LAUNCH_CHECK();
    GBSW_CUDA_TRY(cudaMemcpyAsync(s->h_result, s->result, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    GBSW_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (volume) *volume = s->h_result[0];
    if (wet_volume) *wet_volume = s->h_result[1];
    return s->h_result[2] != 0.0 ? GBSW_ERR_NONFINITE : GBSW_OK;
}

gbsw_status sw_get_state(gbsw_sw *s, float *eta, float *u, float *v, uint8_t *wet)
{
    if (!s) return GBSW_ERR_ARG;
    const int nx = s->p.nx, ny = s->p.ny;
    const size_t dp = (size_t)s->d.pitch * sizeof(float);
    const size_t row = (size_t)nx * sizeof(float);
    const int c = s->cur;
    if (eta)
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(eta, row, s->eta[c], dp, row, ny, cudaMemcpyDeviceToHost, s->stream));
    if (u)
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(u + 1, row + sizeof(float), s->u[c], dp, row, ny,
                                        cudaMemcpyDeviceToHost, s->stream));
    if (v)
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(v + nx, row, s->v[c], dp, row, ny, cudaMemcpyDeviceToHost, s->stream));
    if (wet) {
        dim3 block(32, 8), grid(ceil_div(nx, 32), ceil_div(ny, 8));
        sw_wet_mask_kernel<<<grid, block, 0, s->stream>>>(s->d, s->H, s->eta[c], s->wet);
        GBSW_LAUNCH_CHECK();
        GBSW_CUDA_TRY(cudaMemcpyAsync(wet, s->wet, (size_t)nx * ny, cudaMemcpyDeviceToHost, s->stream));
    }
    GBSW_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (u)
        for (int j = 0; j < ny; ++j) u[(size_t)j * (nx + 1)] = 0.0f;
    if (v)
        for (int i = 0; i < nx; ++i) v[i] = 0.0f;
    return GBSW_OK;
}

gbsw_status sw_set_state(gbsw_sw *s, const float *eta, const float *u, const float *v)
{
    if (!s) return GBSW_ERR_ARG;
    const int nx = s->p.nx, ny = s->p.ny;
    const size_t dp = (size_t)s->d.pitch * sizeof(float);
    const size_t row = (size_t)nx * sizeof(float);
    const int c = s->cur;
    if (eta)
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(s->eta[c], dp, eta, row, row, ny, cudaMemcpyHostToDevice, s->stream));
    if (u) {
        // host columns 1..nx are the faces the device stores; the east wall is forced to 0
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(s->u[c], dp, u + 1, row + sizeof(float), row, ny,
                                        cudaMemcpyHostToDevice, s->stream));
        GBSW_CUDA_TRY(cudaMemset2DAsync(s->u[c] + (nx - 1), dp, 0, sizeof(float), ny, s->stream));
    }
    if (v) {
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(s->v[c], dp, v + nx, row, row, ny, cudaMemcpyHostToDevice, s->stream));
        GBSW_CUDA_TRY(cudaMemsetAsync(s->v[c] + (size_t)(ny - 1) * s->d.pitch, 0, row, s->stream));
    }
    GBSW_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return GBSW_OK;
}

void sw_destroy(gbsw_sw *s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    drop_chunks(s);
    cudaFree(s->H);
    for (int b = 0; b < 2; ++b) {
        cudaFree(s->eta[b]);
        cudaFree(s->u[b]);
        cudaFree(s->v[b]);
    }
    cudaFree(s->partials);
    cudaFree(s->result);
    cudaFree(s->wet);
    if (s->h_result) cudaFreeHost(s->h_result);
    free(s);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Volume reduction that allocates nothing (sw_volume_noalloc).
//
// Some callers cannot call cudaMalloc: applications whose memory pool owns
// the whole device and hands out no raw allocations, and latency-critical
// loops in which a cudaMalloc/cudaFree (which may synchronise the device)
// or an out-of-memory failure in the middle of a run is not acceptable.
// For them the two-pass FP64 volume reduction keeps its per-block partial
// sums in the file-scope array below instead of in context-owned memory.
// The array is SW_VOL_BLOCKS * 3 doubles (24 KB); every GPU that loads the
// library holds it until the process exits.  Each call overwrites all of
// it before reading it, so nothing has to be cleared between calls, but
// all calls share it: calls whose kernels overlap on the GPU (different
// streams, or different host threads) race on it.
// ---------------------------------------------------------------------------
#include <cuda.h>
#include <mutex>

static __device__ __align__(256) double g_sw_volume_scratch[SW_VOL_BLOCKS * 3];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
struct ScratchAddr {
    unsigned long long ctx_id;  // CUDA context the address belongs to (IDs are never reused in a process)
    double *addr;               // device address of g_sw_volume_scratch in that context
};
ScratchAddr g_scratch_addr[kMaxDevices];

// Device address of the scratch array in the current device's context.  In
// host code the array's name is only a host-side stand-in, so the address
// comes from cudaGetSymbolAddress, looked up on the first call in each
// context: once per device, and again if that device's context was
// destroyed and re-created (the module is then loaded anew, at a possibly
// different address).
gbsw_status volume_scratch(double **out)
{
    int dev = 0;
    GBSW_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return GBSW_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    // driver calls through the runtime's entry-point query, so that loading
    // the library does not need the driver library on hosts without a GPU
    using GetCurrentFn = CUresult (*)(CUcontext *);
    using GetIdFn = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
            qa != cudaDriverEntryPointSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
            qb != cudaDriverEntryPointSuccess)
            return GBSW_ERR_CUDA;
        get_current = (GetCurrentFn)a;
        get_id = (GetIdFn)b;
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) {
        // no current context yet: the runtime creates the primary one here
        void *p = nullptr;
        GBSW_CUDA_TRY(cudaGetSymbolAddress(&p, g_sw_volume_scratch));
        if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return GBSW_ERR_CUDA;
    }
    unsigned long long id = 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return GBSW_ERR_CUDA;
    ScratchAddr &e = g_scratch_addr[dev];
    if (!e.addr || e.ctx_id != id) {
        void *p = nullptr;
        GBSW_CUDA_TRY(cudaGetSymbolAddress(&p, g_sw_volume_scratch));
        e.addr = (double *)p;
        e.ctx_id = id;
    }
    *out = e.addr;
    return GBSW_OK;
}

}  // namespace

extern "C" gbsw_status sw_volume_noalloc(int nx, int ny, int pitch, double dx, double dy, double hmin,
                                         const float *H, const float *eta, double *out, void *stream)
{
    if (nx < 1 || ny < 1 || nx > SW_NOALLOC_MAX_SIDE || ny > SW_NOALLOC_MAX_SIDE || pitch < nx)
        return GBSW_ERR_ARG;
    if (!H || !eta || !out || !(dx > 0) || !(dy > 0) || !(hmin >= 0)) return GBSW_ERR_ARG;
    double *scratch = nullptr;
    gbsw_status st = volume_scratch(&scratch);
    if (st != GBSW_OK) return st;
    SWDev d = {};
    d.nx = nx;
    d.ny = ny;
    d.pitch = pitch;
    d.hmin = (float)hmin;
    cudaStream_t s = (cudaStream_t)stream;
    sw_volume_partial_kernel<<<SW_VOL_BLOCKS, SW_VOL_THREADS, 0, s>>>(d, H, eta, scratch);
    GBSW_LAUNCH_CHECK();
    sw_volume_final_kernel<<<1, SW_VOL_THREADS, 0, s>>>(scratch, SW_VOL_BLOCKS, dx * dy, out);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

namespace gbsw {
unsigned long long take_bounds_sw()
{
    unsigned h = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&h, g_sw_bounds, sizeof(h)) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_sw_bounds, &zero, sizeof(zero));
    return h;
}
}  // namespace gbsw

// Batched 2DSW ensemble: many independent shallow-water instances of
// different sizes (the 2DSW step of Sec. 6.2 of arXiv:1711.04471, run as an
// ensemble) advanced by one persistent kernel.
//
// Every instance is cut into (instance, strip, row segment) work items of
// the streaming kernel in sw_stream.cuh.  One cooperative launch runs all
// T-step levels: CTAs pull items of the current level from an atomic
// counter, then meet at a grid barrier (bounded spin; a timeout sets the
// status word and every CTA leaves) before the next level reads what the
// previous one wrote.  Level-0 rows are loaded through L2 (ld.global.cg) so
// that no SM sees a stale L1 line of a buffer rewritten by another SM.
// sw_batch_step captures the launch in a CUDA graph, so an nsteps call is
// one graph launch however many instances there are.
//
// (T, rows per item) are chosen by sw_batch_autotune, which times the
// candidates on the batch itself and can cache the choice in a text file.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "sw_kernels.cuh"
#include "sw_stream.cuh"

using namespace gbsw;

namespace {

struct SWInst {
    SWDev p;
    long long off;  // element offset of the instance in the packed field arrays
};

struct SWItem {
    int inst, strip, r0, r1;
};

struct BatchDev {
    const SWInst *inst;
    const SWItem *items;
    int nitems;
    const float *H;
    float *eta[2], *u[2], *v[2];
    unsigned *counters;  // one work counter per level
    unsigned *bar_count, *bar_gen;
    int *status;
    long long spin_limit;  // polls of a grid-barrier wait before it gives up
};

constexpr long long SPIN_LIMIT = 20000000;  // ~ seconds; a level takes milliseconds
constexpr int VOL_BLOCKS = 16;              // volume partial blocks per instance

// Grid-wide barrier for a cooperative launch.  Returns false (in every
// thread) if the status word is set, e.g. by a timed-out wait.
__device__ bool grid_barrier(const BatchDev &B, unsigned nblocks)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned g = atomicAdd(B.bar_gen, 0u);
        const unsigned arrived = atomicAdd(B.bar_count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(B.bar_count, 0u);
            __threadfence();
            atomicAdd(B.bar_gen, 1u);
        } else {
            long long spins = 0;
            while (atomicAdd(B.bar_gen, 0u) == g) {
                if (++spins > B.spin_limit) {
                    atomicCAS(B.status, DEV_OK, DEV_TIMEOUT);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = atomicAdd(B.status, 0) == DEV_OK;
    }
    __syncthreads();
    return ok;
}

// nlevels levels of T fused steps over every item; buffer parity cur0 at
// the first level.  Cooperative launch, block SWS_THREADS.
template <int T>
__global__ void __launch_bounds__(SWS_THREADS)
sw_batch_kernel(BatchDev B, int nlevels, int cur0)
{
    __shared__ SWStageLines lines[T];
    __shared__ int s_item;
    for (int lv = 0; lv < nlevels; ++lv) {
        // buffer parity of this level, by selects (indexing the parameter's
        // pointer arrays with a run-time index would copy them to local memory)
        const bool odd = ((cur0 + lv) & 1) != 0;
        const float *eta_a = odd ? B.eta[1] : B.eta[0], *u_a = odd ? B.u[1] : B.u[0], *v_a = odd ? B.v[1] : B.v[0];
        float *eta_b = odd ? B.eta[0] : B.eta[1], *u_b = odd ? B.u[0] : B.u[1], *v_b = odd ? B.v[0] : B.v[1];
        for (;;) {
            if (threadIdx.x == 0) s_item = (int)atomicAdd(&B.counters[lv], 1u);
            __syncthreads();
            const int it = s_item;
            __syncthreads();
            if (it >= B.nitems) break;
            const SWItem w = B.items[it];
            const SWInst I = B.inst[w.inst];
            sw_stream_tile<T, SWLoad::L2>(I.p, w.strip, w.r0, w.r1, B.H + I.off, eta_a + I.off, u_a + I.off,
                                          v_a + I.off, eta_b + I.off, u_b + I.off, v_b + I.off, lines);
        }
        if (lv + 1 < nlevels && !grid_barrier(B, gridDim.x)) return;
    }
}

// FP64 volume partials: block (b, m) sums rows b, b + VOL_BLOCKS, ... of
// instance m; the order depends only on the instance's size.
__global__ void __launch_bounds__(SW_VOL_THREADS)
sw_batch_volume_partial(const SWInst *__restrict__ inst, const float *__restrict__ H, const float *__restrict__ eta,
                        double *__restrict__ partials)
{
    __shared__ double red[SW_VOL_THREADS / 32];
    const SWInst I = inst[blockIdx.y];
    const SWDev &p = I.p;
    double s = 0.0, sw = 0.0, bad = 0.0;
    for (int j = blockIdx.x; j < p.ny; j += VOL_BLOCKS) {
        const long long row = I.off + (long long)j * p.pitch;
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
        double *o = partials + 3 * ((long long)blockIdx.y * VOL_BLOCKS + blockIdx.x);
        o[0] = s;
        o[1] = sw;
        o[2] = bad;
    }
}

__global__ void sw_batch_volume_final(const double *__restrict__ partials, const double *__restrict__ area,
                                      double *__restrict__ out)
{
    const int m = blockIdx.x;
    if (threadIdx.x != 0) return;
    double s = 0.0, sw = 0.0, bad = 0.0;
    for (int b = 0; b < VOL_BLOCKS; ++b) {
        const double *o = partials + 3 * ((long long)m * VOL_BLOCKS + b);
        s += o[0];
        sw += o[1];
        bad += o[2];
    }
    out[3 * m] = s * area[m];
    out[3 * m + 1] = sw * area[m];
    out[3 * m + 2] = bad;
}

}  // namespace

struct gbsw_sw_batch {
    int n;
    std::vector<gbsw_sw_params> params;
    std::vector<SWInst> inst_h;
    cudaStream_t stream;
    size_t total;        // elements per packed field
    float *H, *eta[2], *u[2], *v[2];
    SWInst *inst;
    SWItem *items[5];    // work items per fused depth T (strip width depends on T)
    int nitems[5], items_rows[5];
    unsigned *counters, *bar;
    int max_levels;
    int *status;
    double *partials, *area, *vol;
    int cur;
    int T, rows;         // current tiling
    int grid_cache[8];   // co-resident CTAs per T
    std::map<long long, cudaGraphExec_t> graphs;  // key: nsteps * 2 + cur
};

namespace {

void free_graphs(gbsw_sw_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

gbsw_status build_items(gbsw_sw_batch *b, int T, int rows)
{
    if (b->items[T] && b->items_rows[T] == rows) return GBSW_OK;
    const int W = SWS_THREADS - 4 * T;
    std::vector<std::pair<long long, SWItem>> v;
    for (int m = 0; m < b->n; ++m) {
        const int nx = b->params[m].nx, ny = b->params[m].ny;
        for (int s = 0; s * W < nx; ++s)
            for (int r = 0; r < ny; r += rows)
                v.push_back({(long long)nx * ny, SWItem{m, s, r, std::min(ny, r + rows)}});
    }
    // largest instances first, so the dynamic schedule ends with small items
    std::stable_sort(v.begin(), v.end(), [](const auto &x, const auto &y) { return x.first > y.first; });
    std::vector<SWItem> items(v.size());
    for (size_t k = 0; k < v.size(); ++k) items[k] = v[k].second;
    free_graphs(b);  // cached graphs hold the old item pointer
    if (b->items[T]) cudaFree(b->items[T]);
    b->items[T] = nullptr;
    GBSW_CUDA_TRY(cudaMalloc((void **)&b->items[T], items.size() * sizeof(SWItem)));
    GBSW_CUDA_TRY(cudaMemcpy(b->items[T], items.data(), items.size() * sizeof(SWItem), cudaMemcpyHostToDevice));
    b->nitems[T] = (int)items.size();
    b->items_rows[T] = rows;
    return GBSW_OK;
}

template <int T>
gbsw_status launch_batch(gbsw_sw_batch *b, cudaStream_t s, int nlevels, int cur0, unsigned *counters)
{
    int &grid = b->grid_cache[T];
    if (grid == 0) {
        int per_sm = 0;
        GBSW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sw_batch_kernel<T>, SWS_THREADS, 0));
        grid = std::max(1, per_sm) * sm_count();
    }
    BatchDev B;
    B.inst = b->inst;
    B.items = b->items[T];
    B.nitems = b->nitems[T];
    B.H = b->H;
    for (int k = 0; k < 2; ++k) {
        B.eta[k] = b->eta[k];
        B.u[k] = b->u[k];
        B.v[k] = b->v[k];
    }
    B.counters = counters;
    B.bar_count = b->bar;
    B.bar_gen = b->bar + 1;
    B.status = b->status;
    B.spin_limit = fault_injected("sync_timeout") ? 0 : SPIN_LIMIT;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(SWS_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    GBSW_CUDA_TRY(cudaLaunchKernelEx(&cfg, sw_batch_kernel<T>, B, nlevels, cur0));
    return GBSW_OK;
}

gbsw_status launch_levels(gbsw_sw_batch *b, cudaStream_t s, int T, int nlevels, int cur0, unsigned *counters)
{
    switch (T) {
    case 1: return launch_batch<1>(b, s, nlevels, cur0, counters);
    case 2: return launch_batch<2>(b, s, nlevels, cur0, counters);
    case 3: return launch_batch<3>(b, s, nlevels, cur0, counters);
    case 4: return launch_batch<4>(b, s, nlevels, cur0, counters);
    default: return GBSW_ERR_ARG;
    }
}

// Enqueue nsteps as: work counters = 0; one persistent launch of the full
// levels of depth T; one level of the remainder depth.  The item lists of
// both depths must exist.
gbsw_status enqueue_steps(gbsw_sw_batch *b, cudaStream_t s, int nsteps, int cur0)
{
    const int full = nsteps / b->T, tail = nsteps % b->T;
    GBSW_CUDA_TRY(cudaMemsetAsync(b->counters, 0, (size_t)(full + 1) * sizeof(unsigned), s));
    gbsw_status st = GBSW_OK;
    if (full > 0) st = launch_levels(b, s, b->T, full, cur0, b->counters);
    if (st == GBSW_OK && tail > 0) st = launch_levels(b, s, tail, 1, (cur0 + full) & 1, b->counters + full);
    return st;
}

gbsw_status ensure_levels(gbsw_sw_batch *b, int levels)
{
    if (levels <= b->max_levels) return GBSW_OK;
    if (b->counters) cudaFree(b->counters);
    b->counters = nullptr;
    b->max_levels = 0;
    GBSW_CUDA_TRY(cudaMalloc((void **)&b->counters, (size_t)levels * sizeof(unsigned)));
    b->max_levels = levels;
    free_graphs(b);
    return GBSW_OK;
}

}  // namespace

extern "C" {

gbsw_status sw_batch_create(int n, const gbsw_sw_params *params, const double *const *H, const double *const *eta0,
                            void *stream, gbsw_sw_batch **out)
{
    if (n < 1 || !params || !H || !eta0 || !out) return GBSW_ERR_ARG;
    if (fault_injected("alloc")) return GBSW_ERR_OOM;
    gbsw_sw_batch *b = new (std::nothrow) gbsw_sw_batch();
    if (!b) return GBSW_ERR_OOM;
    b->n = n;
    b->stream = (cudaStream_t)stream;
    b->params.assign(params, params + n);
    b->T = 3;
    b->rows = 128;
    long long off = 0;
    std::vector<double> area(n);
    for (int m = 0; m < n; ++m) {
        const gbsw_sw_params &P = params[m];
        if (P.nx < 2 || P.ny < 2 || P.nx > 65536 || P.ny > 65536 || !(P.dx > 0) || !(P.dy > 0) || !(P.dt > 0) ||
            !(P.g > 0) || !(P.eps >= 0 && P.eps <= 1) || !(P.hmin >= 0) || !H[m] || !eta0[m]) {
            delete b;
            return GBSW_ERR_ARG;
        }
        SWInst I = {};
        I.p.nx = P.nx;
        I.p.ny = P.ny;
        I.p.pitch = (int)round_up((size_t)P.nx, 32);
        I.p.gdt_dx = (float)(P.g * P.dt / P.dx);
        I.p.gdt_dy = (float)(P.g * P.dt / P.dy);
        I.p.dt_dx = (float)(P.dt / P.dx);
        I.p.dt_dy = (float)(P.dt / P.dy);
        I.p.q = (float)(0.25 * P.eps);
        I.p.hmin = (float)P.hmin;
        I.off = off;
        off += (long long)I.p.pitch * P.ny;
        b->inst_h.push_back(I);
        area[m] = P.dx * P.dy;
    }
    b->total = (size_t)off;
    // host-side conversion and CFL check per instance
    std::vector<float> h32(b->total, 0.0f), e32(b->total, 0.0f);
    for (int m = 0; m < n; ++m) {
        const gbsw_sw_params &P = params[m];
        const SWInst &I = b->inst_h[m];
        double hmax = 0.0;
        for (int j = 0; j < P.ny; ++j)
            for (int i = 0; i < P.nx; ++i) {
                const size_t k = (size_t)j * P.nx + i;
                const double hv = H[m][k], ev0 = eta0[m][k];
                if (!std::isfinite(hv) || !std::isfinite(ev0)) {
                    delete b;
                    return GBSW_ERR_ARG;
                }
                const double ev = ev0 < -hv ? -hv : ev0;
                hmax = std::max(hmax, hv + ev);
                h32[I.off + (size_t)j * I.p.pitch + i] = (float)hv;
                e32[I.off + (size_t)j * I.p.pitch + i] = (float)ev;
            }
        if (sqrt(P.g * hmax) * P.dt * sqrt(1.0 / (P.dx * P.dx) + 1.0 / (P.dy * P.dy)) > 1.0) {
            delete b;
            return GBSW_ERR_CFL;
        }
    }
    auto fail = [&](gbsw_status st) {
        sw_batch_destroy(b);
        return st;
    };
    const size_t fb = b->total * sizeof(float);
    float **fields[] = {&b->H, &b->eta[0], &b->eta[1], &b->u[0], &b->u[1], &b->v[0], &b->v[1]};
    for (float **f : fields) {
        if (cudaMalloc((void **)f, fb) != cudaSuccess) return fail(GBSW_ERR_OOM);
        if (cudaMemsetAsync(*f, 0, fb, b->stream) != cudaSuccess) return fail(GBSW_ERR_CUDA);
    }
    if (cudaMalloc((void **)&b->inst, n * sizeof(SWInst)) != cudaSuccess ||
        cudaMalloc((void **)&b->bar, 2 * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc((void **)&b->status, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void **)&b->partials, (size_t)n * VOL_BLOCKS * 3 * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&b->area, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&b->vol, (size_t)n * 3 * sizeof(double)) != cudaSuccess)
        return fail(GBSW_ERR_OOM);
    cudaError_t e = cudaMemcpyAsync(b->inst, b->inst_h.data(), n * sizeof(SWInst), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->area, area.data(), n * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->H, h32.data(), fb, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->eta[0], e32.data(), fb, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status, 0, sizeof(int), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        record_cuda_error(e, "sw_batch_create upload", __FILE__, __LINE__);
        return fail(GBSW_ERR_CUDA);
    }
    *out = b;
    return GBSW_OK;
}

gbsw_status sw_batch_set_tiling(gbsw_sw_batch *b, int steps_per_level, int rows_per_item)
{
    if (!b || steps_per_level < 1 || steps_per_level > 4 || rows_per_item < 8 || rows_per_item > 65536)
        return GBSW_ERR_ARG;
    if (b->T != steps_per_level || b->rows != rows_per_item) free_graphs(b);
    b->T = steps_per_level;
    b->rows = rows_per_item;
    return GBSW_OK;
}

gbsw_status sw_batch_get_tiling(gbsw_sw_batch *b, int *steps_per_level, int *rows_per_item)
{
    if (!b) return GBSW_ERR_ARG;
    if (steps_per_level) *steps_per_level = b->T;
    if (rows_per_item) *rows_per_item = b->rows;
    return GBSW_OK;
}

gbsw_status sw_batch_step(gbsw_sw_batch *b, int nsteps)
{
    gbsw::NvtxRange nvtx_range("sw_batch_step");
    if (!b || nsteps < 0) return GBSW_ERR_ARG;
    if (nsteps == 0) return GBSW_OK;
    const int full = nsteps / b->T, tail = nsteps % b->T;
    gbsw_status st = ensure_levels(b, full + 1);
    if (st == GBSW_OK) st = build_items(b, b->T, b->rows);
    if (st == GBSW_OK && tail > 0) st = build_items(b, tail, b->rows);
    if (st != GBSW_OK) return st;
    const long long key = (long long)nsteps * 2 + b->cur;
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        // capture [counters = 0, persistent kernel(s)] once per (nsteps, parity)
        cudaStream_t cs;
        GBSW_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ex = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = enqueue_steps(b, cs, nsteps, b->cur);
            cudaError_t e2 = cudaStreamEndCapture(cs, &g);
            if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess && st == GBSW_OK) e = cudaGraphInstantiate(&ex, g, 0);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess) {
            record_cuda_error(e, "sw_batch graph", __FILE__, __LINE__);
            return GBSW_ERR_CUDA;
        }
        if (st != GBSW_OK) return st;
        it = b->graphs.emplace(key, ex).first;
    }
    GBSW_CUDA_TRY(cudaGraphLaunch(it->second, b->stream));
    b->cur = (b->cur + full + (tail > 0 ? 1 : 0)) & 1;
    return GBSW_OK;
}

/* The same steps as separate launches of the single-grid kernel, one per
 * instance and fused level (the unbatched baseline). */
gbsw_status sw_batch_step_separate(gbsw_sw_batch *b, int nsteps)
{
    if (!b || nsteps < 0) return GBSW_ERR_ARG;
    int left = nsteps;
    while (left > 0) {
        const int T = std::min(left, b->T);
        const int a = b->cur, c = 1 - b->cur;
        static int per_sm[5] = {0, 0, 0, 0, 0};
        if (per_sm[T] == 0) {
            int v = 0;
            switch (T) {
            case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, sw_stream_kernel<1>, SWS_THREADS, 0); break;
            case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, sw_stream_kernel<2>, SWS_THREADS, 0); break;
            case 3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, sw_stream_kernel<3>, SWS_THREADS, 0); break;
            default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, sw_stream_kernel<4>, SWS_THREADS, 0); break;
            }
            per_sm[T] = std::max(1, v);
        }
        for (int m = 0; m < b->n; ++m) {
            const SWInst &I = b->inst_h[m];
            const int W = SWS_THREADS - 4 * T;
            // each launch sized to fill the GPU on its own, as sw_step does
            const int strips = ceil_div(I.p.nx, W);
            int segments = std::max(1, per_sm[T] * sm_count() / strips);
            segments = std::min(segments, std::max(1, I.p.ny / (8 * T)));
            const int rows = ceil_div(I.p.ny, segments);
            dim3 grid(strips, ceil_div(I.p.ny, rows));
#define SEP_LAUNCH(TT)                                                                                         \
    sw_stream_kernel<TT><<<grid, SWS_THREADS, 0, b->stream>>>(I.p, rows, b->H + I.off, b->eta[a] + I.off,          \
                                                              b->u[a] + I.off, b->v[a] + I.off, b->eta[c] + I.off, \
                                                              b->u[c] + I.off, b->v[c] + I.off)
            switch (T) {
            case 1: SEP_LAUNCH(1); break;
            case 2: SEP_LAUNCH(2); break;
            case 3: SEP_LAUNCH(3); break;
            default: SEP_LAUNCH(4); break;
            }
#undef SEP_LAUNCH
        }
        GBSW_LAUNCH_CHECK();
        b->cur = c;
        left -= T;
    }
    return GBSW_OK;
}

gbsw_status sw_batch_volumes(gbsw_sw_batch *b, double *volumes, double *wet_volumes)
{
    gbsw::NvtxRange nvtx_range("sw_batch_volumes");
    if (!b) return GBSW_ERR_ARG;
    sw_batch_volume_partial<<<dim3(VOL_BLOCKS, b->n), SW_VOL_THREADS, 0, b->stream>>>(b->inst, b->H, b->eta[b->cur],
                                                                                  b->partials);
    sw_batch_volume_final<<<b->n, 32, 0, b->stream>>>(b->partials, b->area, b->vol);
    GBSW_LAUNCH_CHECK();
    std::vector<double> h(3 * (size_t)b->n);
    int status = 0;
    GBSW_CUDA_TRY(cudaMemcpyAsync(h.data(), b->vol, h.size() * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    GBSW_CUDA_TRY(cudaMemcpyAsync(&status, b->status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    GBSW_CUDA_TRY(cudaStreamSynchronize(b->stream));
    bool bad = false;
    for (int m = 0; m < b->n; ++m) {
        if (volumes) volumes[m] = h[3 * m];
        if (wet_volumes) wet_volumes[m] = h[3 * m + 1];
        bad = bad || h[3 * m + 2] != 0.0;
    }
    if (status != DEV_OK) return dev_status_to_gbsw(status);
    return bad ? GBSW_ERR_NONFINITE : GBSW_OK;
}

gbsw_status sw_batch_get_state(gbsw_sw_batch *b, int m, float *eta, float *u, float *v)
{
    if (!b || m < 0 || m >= b->n) return GBSW_ERR_ARG;
    const SWInst &I = b->inst_h[m];
    const int nx = I.p.nx, ny = I.p.ny;
    const size_t dp = (size_t)I.p.pitch * sizeof(float), row = (size_t)nx * sizeof(float);
    const int c = b->cur;
    if (eta)
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(eta, row, b->eta[c] + I.off, dp, row, ny, cudaMemcpyDeviceToHost, b->stream));
    if (u)
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(u + 1, row + sizeof(float), b->u[c] + I.off, dp, row, ny,
                                        cudaMemcpyDeviceToHost, b->stream));
    if (v)
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(v + nx, row, b->v[c] + I.off, dp, row, ny, cudaMemcpyDeviceToHost, b->stream));
    GBSW_CUDA_TRY(cudaStreamSynchronize(b->stream));
    if (u)
        for (int j = 0; j < ny; ++j) u[(size_t)j * (nx + 1)] = 0.0f;
    if (v)
        for (int i = 0; i < nx; ++i) v[i] = 0.0f;
    return GBSW_OK;
}

/* Time every (T, rows) candidate on the batch itself (state saved and
 * restored), keep the fastest.  cache_path may be NULL. */
gbsw_status sw_batch_autotune(gbsw_sw_batch *b, int trial_steps, const char *cache_path, int *T_out, int *rows_out)
{
    gbsw::NvtxRange nvtx_range("sw_batch_autotune");
    if (!b || trial_steps < 1) return GBSW_ERR_ARG;
    // cache key: device, instance count and sizes
    cudaDeviceProp prop;
    int dev = 0;
    GBSW_CUDA_TRY(cudaGetDevice(&dev));
    GBSW_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](unsigned long long x) {
        h ^= x;
        h *= 1099511628211ull;
    };
    mix((unsigned long long)b->n);
    for (const auto &p : b->params) {
        mix((unsigned long long)p.nx);
        mix((unsigned long long)p.ny);
    }
    char key[320];
    snprintf(key, sizeof(key), "sw_batch %s %016llx %d", prop.name, h, trial_steps);
    for (char *c = key; *c; ++c)
        if (*c == ' ') *c = '_';  // one whitespace-free token per key
    if (cache_path) {
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char line[512];
            while (fgets(line, sizeof(line), f)) {
                char k[400];
                int T = 0, rows = 0;
                if (sscanf(line, "%399s %d %d", k, &T, &rows) == 3 && strcmp(k, key) == 0) {
                    fclose(f);
                    gbsw_status st = sw_batch_set_tiling(b, T, rows);
                    if (T_out) *T_out = T;
                    if (rows_out) *rows_out = rows;
                    return st;
                }
            }
            fclose(f);
        }
    }
    // save the state
    const size_t fb = b->total * sizeof(float);
    float *save[3] = {nullptr, nullptr, nullptr};
    for (int k = 0; k < 3; ++k) GBSW_CUDA_TRY(cudaMalloc((void **)&save[k], fb));
    const int c0 = b->cur;
    GBSW_CUDA_TRY(cudaMemcpyAsync(save[0], b->eta[c0], fb, cudaMemcpyDeviceToDevice, b->stream));
    GBSW_CUDA_TRY(cudaMemcpyAsync(save[1], b->u[c0], fb, cudaMemcpyDeviceToDevice, b->stream));
    GBSW_CUDA_TRY(cudaMemcpyAsync(save[2], b->v[c0], fb, cudaMemcpyDeviceToDevice, b->stream));
    cudaEvent_t e0, e1;
    GBSW_CUDA_TRY(cudaEventCreate(&e0));
    GBSW_CUDA_TRY(cudaEventCreate(&e1));
    const int Ts[] = {1, 2, 3, 4};
    const int Rs[] = {32, 64, 128, 256};
    float best = 1e30f;
    int bestT = b->T, bestR = b->rows;
    gbsw_status st = GBSW_OK;
    for (int T : Ts)
        for (int R : Rs) {
            st = sw_batch_set_tiling(b, T, R);
            if (st != GBSW_OK) break;
            const int steps = std::max(T, trial_steps / T * T);
            st = sw_batch_step(b, steps);  // warm-up (also builds the graph)
            if (st != GBSW_OK) break;
            cudaEventRecord(e0, b->stream);
            st = sw_batch_step(b, steps);
            cudaEventRecord(e1, b->stream);
            if (st != GBSW_OK) break;
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= (float)steps;
            if (ms < best) {
                best = ms;
                bestT = T;
                bestR = R;
            }
        }
    // restore the state
    b->cur = c0;
    cudaMemcpyAsync(b->eta[c0], save[0], fb, cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(b->u[c0], save[1], fb, cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(b->v[c0], save[2], fb, cudaMemcpyDeviceToDevice, b->stream);
    cudaStreamSynchronize(b->stream);
    for (int k = 0; k < 3; ++k) cudaFree(save[k]);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GBSW_OK) return st;
    st = sw_batch_set_tiling(b, bestT, bestR);
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s %d %d\n", key, bestT, bestR);
            fclose(f);
        }
    }
    if (T_out) *T_out = bestT;
    if (rows_out) *rows_out = bestR;
    return st;
}

void sw_batch_destroy(gbsw_sw_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    free_graphs(b);
    float *fields[] = {b->H, b->eta[0], b->eta[1], b->u[0], b->u[1], b->v[0], b->v[1]};
    for (float *f : fields) cudaFree(f);
    cudaFree(b->inst);
    for (int t = 0; t < 5; ++t) cudaFree(b->items[t]);
    cudaFree(b->counters);
    cudaFree(b->bar);
    cudaFree(b->status);
    cudaFree(b->partials);
    cudaFree(b->area);
    cudaFree(b->vol);
    delete b;
}

}  // extern "C"

namespace gbsw {
unsigned long long take_bounds_batch()
{
    unsigned h = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&h, g_sw_bounds, sizeof(h)) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_sw_bounds, &zero, sizeof(zero));
    return h;
}
}  // namespace gbsw

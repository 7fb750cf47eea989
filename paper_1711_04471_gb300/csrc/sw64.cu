// FP64 2DSW time step (Sec. 6.2 of arXiv:1711.04471) as the paper's three
// map kernels per step: the predictor "dyn" split into its momentum part
// (faces) and its continuity part (cells), then the first-order Shapiro
// filter, with the velocity/state update folded into buffer swaps.
//
// Every operation is written out in the order of the method as stated in
// include/gbsw.h and rounded as written (explicit round-to-nearest FP64
// intrinsics, no multiply-add contraction):
//   u'   = u - ((g dt) (eta_e - eta_c)) / dx, masked by the wet/dry face rule
//   F    = max(u', 0) h_behind + min(u', 0) h_ahead      (two products, one sum)
//   eta* = eta - dt ((F_e - F_w) / dx + (G_n - G_s) / dy)
//   eta+ = (1 - q n) eta*_c + q s on wet cells, q = eps / 4, where n counts
//          the wet neighbours and s sums their eta* in the order east, west,
//          north, south; dry cells keep eta*
// so that the state is a deterministic function of the inputs, bit for bit
// the same on every launch shape.  FP32 is the fast path (sw_step); this
// variant exists for precision: it is the method in FP64 end to end.
//
// Device layout: (ny + 2) rows of `pitch` doubles, cell (i, j) (1-based
// interior, 0 and n + 1 the halo ring) at j * pitch + i; u[j][i] is the
// east face of cell (i, j) (i = 0 .. nx), v[j][i] the north face
// (j = 0 .. ny).  The halo ring of H and eta is 0, so it reads as dry.
#include <math.h>
#include <stdlib.h>

#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"

struct gbsw_sw64 {
    gbsw_sw_params p;
    int pitch;
    cudaStream_t stream;
    double *H;                // (ny+2) x pitch
    double *eta, *eta_new;    // state and the filtered elevation of the step
    double *u, *v, *un, *vn;  // velocities and the predicted ones
    double *es;               // eta* of the step
    double *partials, *result;
    double *h_result;         // pinned, 3 doubles
    std::vector<double> h_H;  // host copy of H (interior, ny x nx) for the wet mask
};

namespace {

constexpr int S64_THREADS = 128;
constexpr int S64_VOL_BLOCKS = 512;

struct S64Dev {
    int nx, ny, pitch;
    double gdt;   // g * dt
    double dx, dy, dt;
    double q;     // eps / 4
    double hmin;
};

__device__ __forceinline__ bool s64_interior(const S64Dev &p, int i, int j)
{
    return i >= 1 && i <= p.nx && j >= 1 && j <= p.ny;
}

// Total depth H + eta of cell (i, j) at the start of the step; 0 off the grid.
__device__ __forceinline__ double s64_depth(const S64Dev &p, const double *H, const double *eta, int i, int j)
{
    const long long c = (long long)j * p.pitch + i;
    return s64_interior(p, i, j) ? __dadd_rn(H[c], eta[c]) : 0.0;
}

__device__ __forceinline__ bool s64_wet(const S64Dev &p, const double *H, const double *eta, int i, int j)
{
    return s64_interior(p, i, j) && s64_depth(p, H, eta, i, j) > p.hmin;
}

// Wet/dry face rule: a is the cell behind the face, b the cell ahead.
__device__ __forceinline__ double s64_mask(double vel, bool wet_a, bool wet_b)
{
    if (wet_a && wet_b) return vel;
    if (wet_a && vel > 0.0) return vel;
    if (wet_b && vel < 0.0) return vel;
    return 0.0;
}

// Upwind volume flux through a face with velocity vel between cells a and b.
__device__ __forceinline__ double s64_flux(double vel, double h_a, double h_b)
{
    const double up = vel > 0.0 ? vel : 0.0;
    const double dn = vel < 0.0 ? vel : 0.0;
    return __dadd_rn(__dmul_rn(up, h_a), __dmul_rn(dn, h_b));
}

// Map 1 ("dyn", momentum): u' on faces (i = 0..nx, j = 1..ny) and v' on
// faces (i = 1..nx, j = 0..ny); wall faces are 0.
// Launch: grid (ceil((nx + 1) / S64_THREADS), ny + 1), block S64_THREADS.
__global__ void __launch_bounds__(S64_THREADS)
sw64_momentum_kernel(S64Dev p, const double *__restrict__ H, const double *__restrict__ eta,
                     const double *__restrict__ u, const double *__restrict__ v, double *__restrict__ un,
                     double *__restrict__ vn)
{
    const int i = blockIdx.x * S64_THREADS + threadIdx.x;
    const int j = blockIdx.y;
    if (i > p.nx || j > p.ny) return;
    const long long c = (long long)j * p.pitch + i;
    if (j >= 1) {
        double val = 0.0;
        if (i >= 1 && i <= p.nx - 1) {
            const double pred = __dsub_rn(u[c], __ddiv_rn(__dmul_rn(p.gdt, __dsub_rn(eta[c + 1], eta[c])), p.dx));
            val = s64_mask(pred, s64_wet(p, H, eta, i, j), s64_wet(p, H, eta, i + 1, j));
        }
        un[c] = val;
    }
    if (i >= 1) {
        double val = 0.0;
        if (j >= 1 && j <= p.ny - 1) {
            const double pred =
                __dsub_rn(v[c], __ddiv_rn(__dmul_rn(p.gdt, __dsub_rn(eta[c + p.pitch], eta[c])), p.dy));
            val = s64_mask(pred, s64_wet(p, H, eta, i, j), s64_wet(p, H, eta, i, j + 1));
        }
        vn[c] = val;
    }
}

// Map 2 ("dyn", continuity): eta* on every interior cell.
// Launch: grid (ceil(nx / S64_THREADS), ny), block S64_THREADS.
__global__ void __launch_bounds__(S64_THREADS)
sw64_continuity_kernel(S64Dev p, const double *__restrict__ H, const double *__restrict__ eta,
                       const double *__restrict__ un, const double *__restrict__ vn, double *__restrict__ es)
{
    const int i = blockIdx.x * S64_THREADS + threadIdx.x + 1;
    const int j = blockIdx.y + 1;
    if (i > p.nx) return;
    const long long c = (long long)j * p.pitch + i;
    const double hc = s64_depth(p, H, eta, i, j);
    const double fe = s64_flux(un[c], hc, s64_depth(p, H, eta, i + 1, j));
    const double fw = s64_flux(un[c - 1], s64_depth(p, H, eta, i - 1, j), hc);
    const double gn = s64_flux(vn[c], hc, s64_depth(p, H, eta, i, j + 1));
    const double gs = s64_flux(vn[c - p.pitch], s64_depth(p, H, eta, i, j - 1), hc);
    const double div = __dadd_rn(__ddiv_rn(__dsub_rn(fe, fw), p.dx), __ddiv_rn(__dsub_rn(gn, gs), p.dy));
    es[c] = __dsub_rn(eta[c], __dmul_rn(p.dt, div));
}

// Map 3 ("shapiro"): masked 5-point filter of eta* on wet cells (wet mask
// of the start of the step).
// Launch: grid (ceil(nx / S64_THREADS), ny), block S64_THREADS.
__global__ void __launch_bounds__(S64_THREADS)
sw64_shapiro_kernel(S64Dev p, const double *__restrict__ H, const double *__restrict__ eta,
                    const double *__restrict__ es, double *__restrict__ eta_new)
{
    const int i = blockIdx.x * S64_THREADS + threadIdx.x + 1;
    const int j = blockIdx.y + 1;
    if (i > p.nx) return;
    const long long c = (long long)j * p.pitch + i;
    if (!s64_wet(p, H, eta, i, j)) {
        eta_new[c] = es[c];
        return;
    }
    const int ni[4] = {i + 1, i - 1, i, i};
    const int nj[4] = {j, j, j + 1, j - 1};
    double count = 0.0, sum = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (s64_wet(p, H, eta, ni[k], nj[k])) {
            count = __dadd_rn(count, 1.0);
            sum = __dadd_rn(sum, es[(long long)nj[k] * p.pitch + ni[k]]);
        }
    eta_new[c] = __dadd_rn(__dmul_rn(__dsub_rn(1.0, __dmul_rn(p.q, count)), es[c]), __dmul_rn(p.q, sum));
}

// FP64 volume partials over rows b, b + S64_VOL_BLOCKS, ... (fixed order).
__global__ void __launch_bounds__(256)
sw64_volume_partial_kernel(S64Dev p, const double *__restrict__ H, const double *__restrict__ eta,
                           double *__restrict__ partials)
{
    __shared__ double red[256 / 32];
    double s = 0.0, sw = 0.0, bad = 0.0;
    for (int j = blockIdx.x + 1; j <= p.ny; j += S64_VOL_BLOCKS)
        for (int i = threadIdx.x + 1; i <= p.nx; i += blockDim.x) {
            const long long c = (long long)j * p.pitch + i;
            if (!isfinite(eta[c])) bad += 1.0;
            const double h = __dadd_rn(H[c], eta[c]);
            s += h;
            if (h > p.hmin) sw += h;
        }
    s = gbsw::block_sum_f64<256 / 32>(s, red);
    sw = gbsw::block_sum_f64<256 / 32>(sw, red);
    bad = gbsw::block_sum_f64<256 / 32>(bad, red);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x] = s;
        partials[3 * blockIdx.x + 1] = sw;
        partials[3 * blockIdx.x + 2] = bad;
    }
}

__global__ void __launch_bounds__(256)
sw64_volume_final_kernel(S64Dev p, const double *__restrict__ partials, double *__restrict__ out)
{
    __shared__ double red[256 / 32];
    double s = 0.0, sw = 0.0, bad = 0.0;
    for (int b = threadIdx.x; b < S64_VOL_BLOCKS; b += blockDim.x) {
        s += partials[3 * b];
        sw += partials[3 * b + 1];
        bad += partials[3 * b + 2];
    }
    s = gbsw::block_sum_f64<256 / 32>(s, red);
    sw = gbsw::block_sum_f64<256 / 32>(sw, red);
    bad = gbsw::block_sum_f64<256 / 32>(bad, red);
    if (threadIdx.x == 0) {
        out[0] = __dmul_rn(__dmul_rn(s, p.dx), p.dy);
        out[1] = __dmul_rn(__dmul_rn(sw, p.dx), p.dy);
        out[2] = bad;
    }
}

S64Dev s64_dev(const gbsw_sw64 *s)
{
    S64Dev d;
    d.nx = s->p.nx;
    d.ny = s->p.ny;
    d.pitch = s->pitch;
    d.gdt = s->p.g * s->p.dt;
    d.dx = s->p.dx;
    d.dy = s->p.dy;
    d.dt = s->p.dt;
    d.q = 0.25 * s->p.eps;
    d.hmin = s->p.hmin;
    return d;
}

}  // namespace

using namespace gbsw;

extern "C" {

void sw64_destroy(gbsw_sw64 *s)
{
    if (!s) return;
    double *bufs[] = {s->H, s->eta, s->eta_new, s->u, s->v, s->un, s->vn, s->es, s->partials, s->result};
    for (double *b : bufs) cudaFree(b);
    if (s->h_result) cudaFreeHost(s->h_result);
    delete s;
}

gbsw_status sw64_create(const gbsw_sw_params *params, const double *H, const double *eta0, void *stream,
                        gbsw_sw64 **out)
{
    if (!params || !H || !eta0 || !out) return GBSW_ERR_ARG;
    const gbsw_sw_params P = *params;
    if (P.nx < 2 || P.ny < 2 || P.nx > (1 << 20) || P.ny > (1 << 20)) return GBSW_ERR_ARG;
    if (!(P.dx > 0) || !(P.dy > 0) || !(P.dt > 0) || !(P.g > 0) || !(P.eps >= 0 && P.eps <= 1) ||
        !(P.hmin >= 0))
        return GBSW_ERR_ARG;
    const size_t n = (size_t)P.nx * (size_t)P.ny;
    std::vector<double> e(n);
    double hmax = 0.0;
    for (size_t k = 0; k < n; ++k) {
        if (!std::isfinite(H[k]) || !std::isfinite(eta0[k])) return GBSW_ERR_ARG;
        e[k] = eta0[k] < -H[k] ? -H[k] : eta0[k];
        hmax = std::max(hmax, H[k] + e[k]);
    }
    const double courant = sqrt(P.g * hmax) * P.dt * sqrt(1.0 / (P.dx * P.dx) + 1.0 / (P.dy * P.dy));
    if (courant > 1.0) return GBSW_ERR_CFL;
    if (fault_injected("alloc")) return GBSW_ERR_OOM;

    gbsw_sw64 *s = new (std::nothrow) gbsw_sw64();
    if (!s) return GBSW_ERR_OOM;
    s->p = P;
    s->pitch = (int)round_up((size_t)P.nx + 2, 16);
    s->stream = (cudaStream_t)stream;
    s->h_H.assign(H, H + n);
    const size_t bytes = (size_t)s->pitch * (size_t)(P.ny + 2) * sizeof(double);
    double **fields[] = {&s->H, &s->eta, &s->eta_new, &s->u, &s->v, &s->un, &s->vn, &s->es};
    for (double **f : fields) {
        cudaError_t err = cudaMalloc((void **)f, bytes);
        if (err == cudaSuccess) err = cudaMemsetAsync(*f, 0, bytes, s->stream);
        if (err != cudaSuccess) {
            record_cuda_error(err, "sw64_create", __FILE__, __LINE__);
            sw64_destroy(s);
            return err == cudaErrorMemoryAllocation ? GBSW_ERR_OOM : GBSW_ERR_CUDA;
        }
    }
    cudaError_t err = cudaMalloc((void **)&s->partials, 3 * S64_VOL_BLOCKS * sizeof(double));
    if (err == cudaSuccess) err = cudaMalloc((void **)&s->result, 3 * sizeof(double));
    if (err == cudaSuccess) err = cudaMallocHost((void **)&s->h_result, 3 * sizeof(double));
    // interior rows 1..ny, columns 1..nx of H and eta
    const size_t dp = (size_t)s->pitch * sizeof(double), hp = (size_t)P.nx * sizeof(double);
    if (err == cudaSuccess)
        err = cudaMemcpy2DAsync(s->H + s->pitch + 1, dp, H, hp, hp, P.ny, cudaMemcpyHostToDevice, s->stream);
    if (err == cudaSuccess)
        err = cudaMemcpy2DAsync(s->eta + s->pitch + 1, dp, e.data(), hp, hp, P.ny, cudaMemcpyHostToDevice, s->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s->stream);
    if (err != cudaSuccess) {
        record_cuda_error(err, "sw64_create", __FILE__, __LINE__);
        sw64_destroy(s);
        return err == cudaErrorMemoryAllocation ? GBSW_ERR_OOM : GBSW_ERR_CUDA;
    }
    *out = s;
    return GBSW_OK;
}

gbsw_status sw64_step(gbsw_sw64 *s, int nsteps)
{
    gbsw::NvtxRange nvtx_range("sw64_step");
    if (!s || nsteps < 0) return GBSW_ERR_ARG;
    const S64Dev d = s64_dev(s);
    const dim3 gf(ceil_div(d.nx + 1, S64_THREADS), d.ny + 1), gc(ceil_div(d.nx, S64_THREADS), d.ny);
    for (int k = 0; k < nsteps; ++k) {
        sw64_momentum_kernel<<<gf, S64_THREADS, 0, s->stream>>>(d, s->H, s->eta, s->u, s->v, s->un, s->vn);
        sw64_continuity_kernel<<<gc, S64_THREADS, 0, s->stream>>>(d, s->H, s->eta, s->un, s->vn, s->es);
        sw64_shapiro_kernel<<<gc, S64_THREADS, 0, s->stream>>>(d, s->H, s->eta, s->es, s->eta_new);
        // update: eta <- eta+, u <- u', v <- v'
        std::swap(s->eta, s->eta_new);
        std::swap(s->u, s->un);
        std::swap(s->v, s->vn);
    }
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status sw64_volume(gbsw_sw64 *s, double *volume, double *wet_volume)
{
    if (!s) return GBSW_ERR_ARG;
    const S64Dev d = s64_dev(s);
    sw64_volume_partial_kernel<<<S64_VOL_BLOCKS, 256, 0, s->stream>>>(d, s->H, s->eta, s->partials);
    sw64_volume_final_kernel<<<1, 256, 0, s->stream>>>(d, s->partials, s->result);
    GBSW_LAUNCH_CHECK();
    GBSW_CUDA_TRY(cudaMemcpyAsync(s->h_result, s->result, 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    GBSW_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (volume) *volume = s->h_result[0];
    if (wet_volume) *wet_volume = s->h_result[1];
    return s->h_result[2] > 0.0 ? GBSW_ERR_NONFINITE : GBSW_OK;
}

gbsw_status sw64_get_state(gbsw_sw64 *s, double *eta, double *u, double *v, uint8_t *wet)
{
    if (!s) return GBSW_ERR_ARG;
    const int nx = s->p.nx, ny = s->p.ny;
    const size_t dp = (size_t)s->pitch * sizeof(double);
    std::vector<double> e;
    if (eta || wet) {
        e.resize((size_t)nx * ny);
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(e.data(), nx * sizeof(double), s->eta + s->pitch + 1, dp,
                                        nx * sizeof(double), ny, cudaMemcpyDeviceToHost, s->stream));
    }
    if (u)  // east faces i = 0..nx of rows 1..ny
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(u, (nx + 1) * sizeof(double), s->u + s->pitch, dp, (nx + 1) * sizeof(double),
                                        ny, cudaMemcpyDeviceToHost, s->stream));
    if (v)  // north faces j = 0..ny of columns 1..nx
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(v, nx * sizeof(double), s->v + 1, dp, nx * sizeof(double), ny + 1,
                                        cudaMemcpyDeviceToHost, s->stream));
    GBSW_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (eta) std::copy(e.begin(), e.end(), eta);
    if (wet)
        for (size_t k = 0; k < e.size(); ++k) wet[k] = (uint8_t)(s->h_H[k] + e[k] > s->p.hmin);
    return GBSW_OK;
}

}  // extern "C"

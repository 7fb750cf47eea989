// Grid transfers of the learned warm start of the pressure solve (the
// network runs on the grid coarsened by f in each direction, where its
// receptive field spans the domain and reaches the smooth error modes that
// set the SOR iteration count):
//
//   r_c = block mean over f^3 cells of r = b - A p_prev,  p_c = block mean of p_prev
//   x   = [r_c / rms(r_c), p_c / rms(p_c)]   (network input, FP32, 2 channels)
//   s   = (f dx)^2 rms(r_c)
//   p  += s * prolong(out)                  (out: the network's coarse output)
//
// A is the 7-point operator of the solve (Neumann at the inflow, ground and
// lid, p = 0 on the outflow face, periodic in y).  prolong interpolates
// trilinearly between coarse cell centres (fine cell i at coarse coordinate
// (i + 1/2)/f - 1/2); beyond the end centres it holds the end value at the
// Neumann walls, takes minus the last value as the ghost past the outflow
// and wraps in y.  Block sums run in FP64 in a fixed order (deterministic).
#include "warmstart.cuh"

namespace gbsw {

namespace {

constexpr int WS_THREADS = 256;
constexpr int WS_PREP_THREADS = 1024;

__device__ __forceinline__ long long ws_at(const WsGrid &g, int i, int j, int k)
{
    return g.off + (long long)(k - 1) * g.sz + (long long)(j - 1) * g.sy + (i - 1);
}

// One group of tpc = min(f^3, 256) threads per coarse cell; the group's
// partial sums meet in a shared-memory tree (fixed order).
__global__ void __launch_bounds__(WS_THREADS)
ws_restrict_kernel(const float *__restrict__ b, const double *__restrict__ p, WsGrid g, double dx, int f,
                   double *__restrict__ rc, double *__restrict__ pc)
{
    __shared__ double sr[WS_THREADS], sp[WS_THREADS];
    const int f3 = f * f * f;
    const int tpc = f3 < WS_THREADS ? f3 : WS_THREADS;
    const int ncx = g.nx / f, ncy = g.ny / f, ncz = g.nz / f;
    const long long nc = (long long)ncx * ncy * ncz;
    const long long q = (long long)blockIdx.x * (WS_THREADS / tpc) + threadIdx.x / tpc;
    const int lane = threadIdx.x % tpc;
    const double r2 = 1.0 / (dx * dx);
    double accr = 0.0, accp = 0.0;
    if (q < nc) {
        const int I = (int)(q % ncx), J = (int)((q / ncx) % ncy), K = (int)(q / ((long long)ncx * ncy));
        auto P = [&](int i, int j, int k) -> double {
            if (i < 1 || i > g.nx || k < 1 || k > g.nz) return 0.0;
            return p[ws_at(g, i, j, k)];
        };
        for (int t = lane; t < f3; t += tpc) {
            const int i = I * f + t % f + 1, j = J * f + (t / f) % f + 1, k = K * f + t / (f * f) + 1;
            const int jm = j == 1 ? g.ny : j - 1, jp = j == g.ny ? 1 : j + 1;
            const double diag = 6.0 - (i == 1) - (k == 1) - (k == g.nz) + (i == g.nx);
            const double pv = P(i, j, k);
            const double nb = (P(i - 1, j, k) + P(i + 1, j, k)) + (P(i, jm, k) + P(i, jp, k)) +
                              (P(i, j, k - 1) + P(i, j, k + 1));
            accr += (double)b[ws_at(g, i, j, k)] - (nb - diag * pv) * r2;
            accp += pv;
        }
    }
    sr[threadIdx.x] = accr;
    sp[threadIdx.x] = accp;
    __syncthreads();
    for (int h = tpc / 2; h > 0; h >>= 1) {
        if (lane < h) {
            sr[threadIdx.x] += sr[threadIdx.x + h];
            sp[threadIdx.x] += sp[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (lane == 0 && q < nc) {
        rc[q] = sr[threadIdx.x] / f3;
        pc[q] = sp[threadIdx.x] / f3;
    }
}

// Single CTA: the two RMS values, the scaled input and s.
__global__ void __launch_bounds__(WS_PREP_THREADS)
ws_prepare_kernel(const double *__restrict__ rc, const double *__restrict__ pc, long long nc, double hc2,
                  float *__restrict__ xin, double *__restrict__ scale)
{
    __shared__ double red[WS_PREP_THREADS / 32];
    __shared__ double rms[2];
    double a = 0.0, c = 0.0;
    for (long long q = threadIdx.x; q < nc; q += WS_PREP_THREADS) {
        a += rc[q] * rc[q];
        c += pc[q] * pc[q];
    }
    a = block_sum_f64<WS_PREP_THREADS / 32>(a, red);
    c = block_sum_f64<WS_PREP_THREADS / 32>(c, red);
    if (threadIdx.x == 0) {
        rms[0] = sqrt(a / (double)nc);
        rms[1] = sqrt(c / (double)nc);
        *scale = hc2 * rms[0];
    }
    __syncthreads();
    const double rr = rms[0], rp = rms[1];
    for (long long q = threadIdx.x; q < nc; q += WS_PREP_THREADS) {
        xin[2 * q] = rr > 0.0 ? (float)(rc[q] / rr) : 0.0f;
        xin[2 * q + 1] = rp > 0.0 ? (float)(pc[q] / rp) : 0.0f;
    }
}

__global__ void __launch_bounds__(WS_THREADS)
ws_prolong_kernel(const float *__restrict__ out, WsGrid g, int f, const double *__restrict__ scale,
                  double *__restrict__ p)
{
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const double s = *scale;
    const int i = (int)(v % g.nx), j = (int)((v / g.nx) % g.ny), k = (int)(v / ((long long)g.nx * g.ny));
    const int ncx = g.nx / f, ncy = g.ny / f, ncz = g.nz / f;
    const double inv = 1.0 / f;
    // x: held at the inflow, antisymmetric ghost past the outflow
    const double X = fmax((i + 0.5) * inv - 0.5, 0.0);
    const int i0 = min((int)floor(X), ncx - 1);
    const double wx = X - i0;
    int i1 = i0 + 1;
    double sx = 1.0;
    if (i1 >= ncx) {
        i1 = ncx - 1;
        sx = -1.0;
    }
    // y: periodic
    const double Y = (j + 0.5) * inv - 0.5;
    const int jf = (int)floor(Y);
    const double wy = Y - jf;
    const int j0 = (jf + ncy) % ncy, j1 = (jf + 1) % ncy;
    // z: held at the ground and the lid
    const double Z = fmin(fmax((k + 0.5) * inv - 0.5, 0.0), ncz - 1.0);
    const int k0 = min((int)floor(Z), ncz - 1);
    const double wz = Z - k0;
    const int k1 = min(k0 + 1, ncz - 1);
    auto C = [&](int kk, int jj, int ii) { return (double)out[((long long)kk * ncy + jj) * ncx + ii]; };
    auto line = [&](int kk, int jj) { return (1.0 - wx) * C(kk, jj, i0) + wx * sx * C(kk, jj, i1); };
    const double c0 = (1.0 - wy) * line(k0, j0) + wy * line(k0, j1);
    const double c1 = (1.0 - wy) * line(k1, j0) + wy * line(k1, j1);
    p[ws_at(g, i + 1, j + 1, k + 1)] += s * ((1.0 - wz) * c0 + wz * c1);
}

}  // namespace

bool ws_factor_ok(int nx, int ny, int nz, int f)
{
    if (f < 1 || f > 64 || (f & (f - 1))) return false;
    return nx % f == 0 && ny % f == 0 && nz % f == 0;
}

gbsw_status launch_ws_restrict(const float *b, const double *p, const WsGrid &g, double dx, int f, double *rc,
                               double *pc, cudaStream_t s)
{
    if (!ws_factor_ok(g.nx, g.ny, g.nz, f)) return GBSW_ERR_ARG;
    const long long nc = (long long)(g.nx / f) * (g.ny / f) * (g.nz / f);
    const int f3 = f * f * f;
    const int per_cta = WS_THREADS / (f3 < WS_THREADS ? f3 : WS_THREADS);
    ws_restrict_kernel<<<(unsigned)((nc + per_cta - 1) / per_cta), WS_THREADS, 0, s>>>(b, p, g, dx, f, rc, pc);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status launch_ws_prepare(const double *rc, const double *pc, long long nc, double hc2, float *xin,
                              double *scale, cudaStream_t s)
{
    ws_prepare_kernel<<<1, WS_PREP_THREADS, 0, s>>>(rc, pc, nc, hc2, xin, scale);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

gbsw_status launch_ws_prolong(const float *out, const WsGrid &g, int f, const double *scale, double *p,
                              cudaStream_t s)
{
    if (!ws_factor_ok(g.nx, g.ny, g.nz, f)) return GBSW_ERR_ARG;
    const long long n = (long long)g.nx * g.ny * g.nz;
    ws_prolong_kernel<<<(unsigned)((n + WS_THREADS - 1) / WS_THREADS), WS_THREADS, 0, s>>>(out, g, f, scale, p);
    GBSW_LAUNCH_CHECK();
    return GBSW_OK;
}

}  // namespace gbsw

using namespace gbsw;

namespace {

WsGrid dense_grid(int nx, int ny, int nz)
{
    WsGrid g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.sy = nx;
    g.sz = (long long)nx * ny;
    g.off = 0;
    return g;
}

}  // namespace

extern "C" gbsw_status warm_start_features(int nx, int ny, int nz, double dx, int f, const double *p, const float *b,
                                           float *x, double *scale, void *stream)
{
    if (nx < 2 || ny < 2 || nz < 2 || !(dx > 0) || !p || !b || !x || !scale || !ws_factor_ok(nx, ny, nz, f))
        return GBSW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const long long nc = (long long)(nx / f) * (ny / f) * (nz / f);
    double *buf = nullptr;
    gbsw_status st = GBSW_OK;
    cudaError_t e = cudaMalloc((void **)&buf, (size_t)(2 * nc + 1) * sizeof(double));
    if (e != cudaSuccess) {
        record_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        return GBSW_ERR_OOM;
    }
    const WsGrid g = dense_grid(nx, ny, nz);
    st = launch_ws_restrict(b, p, g, dx, f, buf, buf + nc, s);
    if (st == GBSW_OK) st = launch_ws_prepare(buf, buf + nc, nc, (f * dx) * (f * dx), x, buf + 2 * nc, s);
    if (st == GBSW_OK) {
        if ((e = cudaMemcpyAsync(scale, buf + 2 * nc, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess) {
            record_cuda_error(e, "warm_start_features", __FILE__, __LINE__);
            st = GBSW_ERR_CUDA;
        }
    }
    cudaFree(buf);
    return st;
}

extern "C" gbsw_status warm_start_apply(int nx, int ny, int nz, int f, const float *out, double scale, double *p,
                                        void *stream)
{
    if (nx < 2 || ny < 2 || nz < 2 || !out || !p || !ws_factor_ok(nx, ny, nz, f)) return GBSW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    double *d = nullptr;
    cudaError_t e = cudaMalloc((void **)&d, sizeof(double));
    if (e != cudaSuccess) {
        record_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        return GBSW_ERR_OOM;
    }
    gbsw_status st = GBSW_OK;
    if ((e = cudaMemcpyAsync(d, &scale, sizeof(double), cudaMemcpyHostToDevice, s)) != cudaSuccess) {
        record_cuda_error(e, "warm_start_apply", __FILE__, __LINE__);
        st = GBSW_ERR_CUDA;
    }
    if (st == GBSW_OK) st = launch_ws_prolong(out, dense_grid(nx, ny, nz), f, d, p, s);
    if (st == GBSW_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) {
        record_cuda_error(e, "warm_start_apply", __FILE__, __LINE__);
        st = GBSW_ERR_CUDA;
    }
    cudaFree(d);
    return st;
}

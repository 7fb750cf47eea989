// Grid transfers of the learned warm start of the pressure solve (the
// network runs on the grid coarsened by f in each direction, where its
// receptive field spans the domain and reaches the smooth error modes that
// set the SOR iteration count):
//
//   r_c = prolong^T r / f^3 for r = b - A p_prev,  p_c = prolong^T p_prev / f^3
//   x   = [r_c / rms(r_c), p_c / rms(p_c)]   (network input, FP32, 2 channels)
//   s   = (f dx)^2 rms(r_c)
//   p  += s * prolong(out)                  (out: the network's coarse output)
//
// A is the 7-point operator of the solve (Neumann at the inflow, ground and
// lid, p = 0 on the outflow face, periodic in y).  prolong interpolates
// trilinearly between coarse cell centres (fine cell i at coarse coordinate
// (i + 1/2)/f - 1/2); beyond the end centres it holds the end value at the
// Neumann walls, takes minus the last value as the ghost past the outflow
// and wraps in y.  The restriction (full weighting, the prolongation's
// adjoint) keeps the residual's projection on the slowest mode, which sets
// that mode's amplitude in the increment; it runs as three separable passes
// in FP64, each sum in a fixed order (deterministic).
#include "warmstart.cuh"

namespace gbsw {

// Out-of-range index count of the bounds-checked debug build.
static __device__ unsigned g_ws_bounds;

unsigned long long take_bounds_ws()
{
    unsigned h = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&h, g_ws_bounds, sizeof(h)) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_ws_bounds, &zero, sizeof(zero));
    return h;
}

// Index test of the bounds-checked build on a field of the grid; always
// true in the product build.
#define WS_OK(g, c) GBSW_INBOUNDS((c), (g).extent, &g_ws_bounds)

namespace {

constexpr int WS_THREADS = 256;
constexpr int WS_PREP_THREADS = 1024;

__device__ __forceinline__ long long ws_at(const WsGrid &g, int i, int j, int k)
{
    return g.off + (long long)(k - 1) * g.sz + (long long)(j - 1) * g.sy + (i - 1);
}

// Weight of coarse index I in the interpolation at fine index i along one
// axis (the prolongation's rule): 0 = end values held (Neumann walls),
// 1 = periodic, 2 = held at the start, antisymmetric ghost past the end
// (outflow).  Full weighting applies the same weights transposed.
__device__ __forceinline__ double ws_weight(int i, int I, int nc, double inv, int rule)
{
    double X = (i + 0.5) * inv - 0.5;
    if (rule == 1) {
        const int i0 = (int)floor(X);
        const double w = X - i0;
        const int c0 = ((i0 % nc) + nc) % nc, c1 = (c0 + 1) % nc;
        return (c0 == I ? 1.0 - w : 0.0) + (c1 == I ? w : 0.0);
    }
    X = fmax(X, 0.0);
    if (rule == 0) X = fmin(X, nc - 1.0);
    const int i0 = min((int)floor(X), nc - 1);
    const double w = X - i0;
    if (i0 + 1 < nc) return (i0 == I ? 1.0 - w : 0.0) + (i0 + 1 == I ? w : 0.0);
    return I == nc - 1 ? (rule == 2 ? 1.0 - 2.0 * w : 1.0) : 0.0;
}

// The residual r = b - A p of every fine cell, in FP64, once (the x pass
// reads it for both coarse cells a fine cell feeds).  r2 = 1/dx^2 from the
// host; the diagonal 6 - [i == 1] - [k == 1] - [k == nz] + [i == nx] is
// picked by integer selects (no FP64 operation).  r: dense (nz, ny, nx).
__global__ void __launch_bounds__(WS_THREADS)
ws_resid_kernel(const float *__restrict__ b, const double *__restrict__ p, WsGrid g, double r2,
                double *__restrict__ r)
{
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int i = (int)(q % g.nx) + 1;
    const int j = (int)((q / g.nx) % g.ny) + 1;
    const int k = (int)(q / ((long long)g.nx * g.ny)) + 1;
    const int jm = j == 1 ? g.ny : j - 1, jp = j == g.ny ? 1 : j + 1;
    auto P = [&](int ii, int jj, int kk) -> double {
        if (ii < 1 || ii > g.nx || kk < 1 || kk > g.nz || !WS_OK(g, ws_at(g, ii, jj, kk))) return 0.0;
        return p[ws_at(g, ii, jj, kk)];
    };
    const int dci = 6 - (i == 1) - (k == 1) - (k == g.nz) + (i == g.nx);
    const double diag = dci == 6 ? 6.0 : (dci == 5 ? 5.0 : (dci == 7 ? 7.0 : (dci == 4 ? 4.0 : 3.0)));
    const double pv = P(i, j, k);
    const double nb = (P(i - 1, j, k) + P(i + 1, j, k)) + (P(i, jm, k) + P(i, jp, k)) +
                      (P(i, j, k - 1) + P(i, j, k + 1));
    const double bc = WS_OK(g, ws_at(g, i, j, k)) ? (double)b[ws_at(g, i, j, k)] : 0.0;
    r[q] = bc - (nb - diag * pv) * r2;
}

// Table of the full-weighting weights along one axis of n fine cells and
// nc = n / f coarse cells: entry I * 2f + o is the weight of fine cell
// I f - f/2 + o in coarse cell I (0 outside the axis), by ws_weight.
__global__ void ws_wtab_kernel(int n, int nc, int f, int rule, double *__restrict__ wtab)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nc * 2 * f) return;
    const int I = idx / (2 * f), i0 = I * f - f / 2 + idx % (2 * f);
    wtab[idx] = (i0 >= 0 && i0 < n) ? ws_weight(i0, I, nc, 1.0 / f, rule) : 0.0;
}

// Full weighting, pass x: ar/ap (nz, ny, ncx) = weighted sums along x of
// the residual r (dense, from ws_resid_kernel) and of p.  Coarse I draws on
// the 2f fine cells [I f - f/2, I f + 3f/2) (clipped); the sums run in a
// fixed order, with the weights of ws_wtab_kernel (rule 2).
__global__ void __launch_bounds__(WS_THREADS)
ws_fw_x_kernel(const double *__restrict__ r, const double *__restrict__ p, WsGrid g, int f,
               const double *__restrict__ wtab, double *__restrict__ ar, double *__restrict__ ap)
{
    const int ncx = g.nx / f;
    const long long n = (long long)g.nz * g.ny * ncx;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int I = (int)(q % ncx);
    const int j = (int)((q / ncx) % g.ny) + 1;
    const int k = (int)(q / ((long long)ncx * g.ny)) + 1;
    const long long row = ((long long)(k - 1) * g.ny + (j - 1)) * g.nx;
    double sr = 0.0, sp = 0.0;
    const int base = I * f - f / 2;
    const int lo = max(base, 0), hi = min(I * f + (3 * f) / 2, g.nx);
    for (int i0 = lo; i0 < hi; ++i0) {
        const double w = wtab[I * 2 * f + (i0 - base)];
        if (w == 0.0) continue;
        sr += w * r[row + i0];
        sp += w * (WS_OK(g, ws_at(g, i0 + 1, j, k)) ? p[ws_at(g, i0 + 1, j, k)] : 0.0);
    }
    ar[q] = sr;
    ap[q] = sp;
}

// Pass y (periodic): (nz, ny, ncx) -> (nz, ncy, ncx).
__global__ void __launch_bounds__(WS_THREADS)
ws_fw_y_kernel(const double *__restrict__ ar, const double *__restrict__ ap, int nz, int ny, int ncx, int f,
               double *__restrict__ br, double *__restrict__ bp)
{
    const int ncy = ny / f;
    const long long n = (long long)nz * ncy * ncx;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int I = (int)(q % ncx), J = (int)((q / ncx) % ncy), k = (int)(q / ((long long)ncx * ncy));
    const double inv = 1.0 / f;
    double sr = 0.0, sp = 0.0;
    for (int j0 = J * f - f / 2; j0 < J * f + (3 * f) / 2; ++j0) {
        const int jw = ((j0 % ny) + ny) % ny;
        const double w = ws_weight(jw, J, ncy, inv, 1);
        if (w == 0.0) continue;
        const long long src = ((long long)k * ny + jw) * ncx + I;
        sr += w * ar[src];
        sp += w * ap[src];
    }
    br[q] = sr;
    bp[q] = sp;
}

// Pass z (Neumann) and the 1/f^3 normalisation: (nz, ncy, ncx) -> rc, pc.
__global__ void __launch_bounds__(WS_THREADS)
ws_fw_z_kernel(const double *__restrict__ br, const double *__restrict__ bp, int nz, int ncy, int ncx, int f,
               double *__restrict__ rc, double *__restrict__ pc)
{
    const int ncz = nz / f;
    const long long n = (long long)ncz * ncy * ncx;
    const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int I = (int)(q % ncx), J = (int)((q / ncx) % ncy), K = (int)(q / ((long long)ncx * ncy));
    const double inv = 1.0 / f;
    double sr = 0.0, sp = 0.0;
    const int lo = max(K * f - f / 2, 0), hi = min(K * f + (3 * f) / 2, nz);
    for (int k0 = lo; k0 < hi; ++k0) {
        const double w = ws_weight(k0, K, ncz, inv, 0);
        if (w == 0.0) continue;
        const long long src = ((long long)k0 * ncy + J) * ncx + I;
        sr += w * br[src];
        sp += w * bp[src];
    }
    const double norm = inv * inv * inv;
    rc[q] = sr * norm;
    pc[q] = sp * norm;
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

// p += s * prolong(out) on the fine cells of column (i, j), planes
// WS_KCH ch .. WS_KCH ch + WS_KCH - 1 (one thread; grid (columns / block,
// chunks)).  The block forms the chunk's z weights once in shared memory;
// the x and y interpolation of the two coarse planes k0, k1 (c0, c1) is
// formed again only when they change along the column; each cell then
// takes the z interpolation: the same expressions in the same order as a
// cell-by-cell evaluation.
constexpr int WS_KCH = 8;
__global__ void __launch_bounds__(WS_THREADS)
ws_prolong_kernel(const float *__restrict__ out, WsGrid g, int f, const double *__restrict__ scale,
                  double *__restrict__ p)
{
    __shared__ double zw[WS_KCH];
    __shared__ int zk0[WS_KCH], zk1[WS_KCH];
    const int ch = blockIdx.y;
    const int ncx = g.nx / f, ncy = g.ny / f, ncz = g.nz / f;
    const double inv = 1.0 / f;
    if (threadIdx.x < WS_KCH) {
        // z: held at the ground and the lid
        const int k = ch * WS_KCH + threadIdx.x;
        const double Z = fmin(fmax((k + 0.5) * inv - 0.5, 0.0), ncz - 1.0);
        const int k0 = min((int)floor(Z), ncz - 1);
        zw[threadIdx.x] = Z - k0;
        zk0[threadIdx.x] = k0;
        zk1[threadIdx.x] = min(k0 + 1, ncz - 1);
    }
    __syncthreads();
    const long long n = (long long)g.nx * g.ny;
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const double s = *scale;
    const int i = (int)(v % g.nx), j = (int)(v / g.nx);
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
    auto C = [&](int kk, int jj, int ii) { return (double)out[((long long)kk * ncy + jj) * ncx + ii]; };
    auto line = [&](int kk, int jj) { return (1.0 - wx) * C(kk, jj, i0) + wx * sx * C(kk, jj, i1); };
    int kc0 = -1, kc1 = -1;
    double c0 = 0.0, c1 = 0.0;
    const int kend = min((ch + 1) * WS_KCH, g.nz);
    for (int k = ch * WS_KCH; k < kend; ++k) {
        const int e = k - ch * WS_KCH;
        const int k0 = zk0[e], k1 = zk1[e];
        const double wz = zw[e];
        if (k0 != kc0 || k1 != kc1) {
            c0 = (1.0 - wy) * line(k0, j0) + wy * line(k0, j1);
            c1 = (1.0 - wy) * line(k1, j0) + wy * line(k1, j1);
            kc0 = k0;
            kc1 = k1;
        }
        if (WS_OK(g, ws_at(g, i + 1, j + 1, k + 1))) p[ws_at(g, i + 1, j + 1, k + 1)] += s * ((1.0 - wz) * c0 + wz * c1);
    }
}

}  // namespace

bool ws_factor_ok(int nx, int ny, int nz, int f)
{
    if (f < 1 || f > 64 || (f & (f - 1))) return false;
    return nx % f == 0 && ny % f == 0 && nz % f == 0;
}

size_t ws_scratch_doubles(int nx, int ny, int nz, int f)
{
    const size_t ncx = (size_t)(nx / f), ncy = (size_t)(ny / f);
    // residual, x-pass sums, y-pass sums, x weight table
    return (size_t)nx * ny * nz + 2 * (size_t)nz * ny * ncx + 2 * (size_t)nz * ncy * ncx + 2 * (size_t)nx;
}

gbsw_status launch_ws_restrict(const float *b, const double *p, const WsGrid &g, double dx, int f, double *scratch,
                               double *rc, double *pc, cudaStream_t s)
{
    if (!ws_factor_ok(g.nx, g.ny, g.nz, f)) return GBSW_ERR_ARG;
    const int ncx = g.nx / f, ncy = g.ny / f;
    const long long n0 = (long long)g.nx * g.ny * g.nz;
    const long long n1 = (long long)g.nz * g.ny * ncx, n2 = (long long)g.nz * ncy * ncx;
    const long long nc = (long long)(g.nz / f) * ncy * ncx;
    double *res = scratch, *ar = res + n0, *ap = ar + n1, *br = ap + n1, *bp = br + n2, *wx = bp + n2;
    auto blocks = [](long long n) { return (unsigned)((n + WS_THREADS - 1) / WS_THREADS); };
    ws_resid_kernel<<<blocks(n0), WS_THREADS, 0, s>>>(b, p, g, 1.0 / (dx * dx), res);
    ws_wtab_kernel<<<blocks(2LL * g.nx), WS_THREADS, 0, s>>>(g.nx, ncx, f, 2, wx);
    ws_fw_x_kernel<<<blocks(n1), WS_THREADS, 0, s>>>(res, p, g, f, wx, ar, ap);
    ws_fw_y_kernel<<<blocks(n2), WS_THREADS, 0, s>>>(ar, ap, g.nz, g.ny, ncx, f, br, bp);
    ws_fw_z_kernel<<<blocks(nc), WS_THREADS, 0, s>>>(br, bp, g.nz, ncy, ncx, f, rc, pc);
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
    const long long n = (long long)g.nx * g.ny;
    const dim3 grid((unsigned)((n + WS_THREADS - 1) / WS_THREADS), (unsigned)((g.nz + WS_KCH - 1) / WS_KCH));
    ws_prolong_kernel<<<grid, WS_THREADS, 0, s>>>(out, g, f, scale, p);
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
    g.extent = (long long)nx * ny * nz;
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
    cudaError_t e =
        cudaMalloc((void **)&buf, (size_t)(2 * nc + 1 + ws_scratch_doubles(nx, ny, nz, f)) * sizeof(double));
    if (e != cudaSuccess) {
        record_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        return GBSW_ERR_OOM;
    }
    const WsGrid g = dense_grid(nx, ny, nz);
    st = launch_ws_restrict(b, p, g, dx, f, buf + 2 * nc + 1, buf, buf + nc, s);
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

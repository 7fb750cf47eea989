// UFLES time step (Sec. 6.3.1 of arXiv:1711.04471): velnw -> bondv1 ->
// velfg -> feedbf -> les -> adam -> press, on the GPU.
//
// Kernels per step:
//   les_velnw_kernel      u = u* - dt grad p                     (velnw)
//   les_bc_{x,y,z}_kernel inflow face and ghost layer            (bondv1)
//   les_nut_kernel        Smagorinsky nu_t incl. ghost layer     (les, part 1)
//   les_predict_kernel    advection + Goldstein forcing + viscous
//                         stress divergence + Adams-Bashforth    (velfg, feedbf, les, adam)
//   les_rhs_kernel        b = div(u*) / dt                       (press, right-hand side)
//   PoissonSolver         red-black SOR to the FP64 tolerance    (press)
// The paper's compiler emitted 29 map and 4 reduction kernels for this
// loop; here velfg, feedbf, the viscous terms and adam are one kernel.
//
// Layout: every field is a (nz+2) x (ny+2) x pitch FP32 array with one
// ghost layer (pitch = nx+2 rounded up to 32), cell (i,j,k) at
// k*plane + j*pitch + i, u on east faces, v on north faces, w on top faces
// (the conventions of the FP64 oracle); the pressure is the solver's FP64
// p_hi in the same layout.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "poisson.cuh"
#include "unet_ops.cuh"
#include "warmstart.cuh"

using namespace gbsw;

namespace {

struct LDev {
    PDims d;
    float dt, rdx, c_grad;   // c_grad = dt/dx
    float l2;                // (cs dx)^2
    float nu, alpha, beta;
    float rdxdt;             // 1/(dx dt)
};

enum : uint8_t { FACE_U = 1, FACE_V = 2, FACE_W = 4 };

__device__ __forceinline__ long long L(const PDims &d, int i, int j, int k)
{
    return (long long)k * d.plane + (long long)j * d.pitch + i;
}

// velnw: projection with the previous pressure, interior faces only.
__global__ void les_velnw_kernel(LDev q, const double *__restrict__ p, float *__restrict__ u, float *__restrict__ v,
                                 float *__restrict__ w)
{
    const PDims &d = q.d;
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y + 1, k = blockIdx.z + 1;
    if (i > d.nx) return;
    const long long c = L(d, i, j, k);
    const double pc = p[c];
    const double pe = (i < d.nx) ? p[c + 1] : -pc;
    const double pn = p[L(d, i, (j < d.ny) ? j + 1 : 1, k)];
    u[c] -= q.c_grad * (float)(pe - pc);
    v[c] -= q.c_grad * (float)(pn - pc);
    if (k < d.nz) w[c] -= q.c_grad * (float)(p[c + d.plane] - pc);
}

// bondv1, x planes: inflow profile, v = w = 0 at the inflow, zero gradient
// at the outflow.  grid (ceil(ny/128), nz), block 128.
__global__ void les_bc_x_kernel(LDev q, const float *__restrict__ uin, float *u, float *v, float *w)
{
    const PDims &d = q.d;
    const int j = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int k = blockIdx.y + 1;
    if (j > d.ny) return;
    const long long c0 = L(d, 0, j, k), cn = L(d, d.nx, j, k);
    u[c0] = uin[k];
    u[cn + 1] = u[cn];
    v[c0] = -v[c0 + 1];
    v[cn + 1] = v[cn];
    w[c0] = -w[c0 + 1];
    w[cn + 1] = w[cn];
}

// bondv1, y planes: periodic.  grid (ceil((nx+2)/128), nz), block 128.
__global__ void les_bc_y_kernel(LDev q, float *u, float *v, float *w)
{
    const PDims &d = q.d;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y + 1;
    if (i > d.nx + 1) return;
    const long long s0 = L(d, i, 0, k), s1 = L(d, i, 1, k), sn = L(d, i, d.ny, k), sn1 = L(d, i, d.ny + 1, k);
    u[s0] = u[sn];
    u[sn1] = u[s1];
    v[s0] = v[sn];
    v[sn1] = v[s1];
    w[s0] = w[sn];
    w[sn1] = w[s1];
}

// bondv1, z planes: no slip at the ground, free slip at the lid.
// grid (ceil((nx+2)/128), ny+2), block 128.
__global__ void les_bc_z_kernel(LDev q, float *u, float *v, float *w)
{
    const PDims &d = q.d;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i > d.nx + 1) return;
    const long long g0 = L(d, i, j, 0), g1 = g0 + d.plane;
    const long long t0 = L(d, i, j, d.nz), t1 = t0 + d.plane;
    u[g0] = -u[g1];
    v[g0] = -v[g1];
    w[g0] = 0.0f;
    u[t1] = u[t0];
    v[t1] = v[t0];
    w[t0] = 0.0f;
    w[t1] = 0.0f;
}

__device__ __forceinline__ float s12e(const PDims &d, float rdx, const float *u, const float *v, int i, int j, int k)
{
    return 0.5f * ((u[L(d, i, j + 1, k)] - u[L(d, i, j, k)]) + (v[L(d, i + 1, j, k)] - v[L(d, i, j, k)])) * rdx;
}
__device__ __forceinline__ float s13e(const PDims &d, float rdx, const float *u, const float *w, int i, int j, int k)
{
    return 0.5f * ((u[L(d, i, j, k + 1)] - u[L(d, i, j, k)]) + (w[L(d, i + 1, j, k)] - w[L(d, i, j, k)])) * rdx;
}
__device__ __forceinline__ float s23e(const PDims &d, float rdx, const float *v, const float *w, int i, int j, int k)
{
    return 0.5f * ((v[L(d, i, j, k + 1)] - v[L(d, i, j, k)]) + (w[L(d, i, j + 1, k)] - w[L(d, i, j, k)])) * rdx;
}

// les, part 1: nu_t = (cs dx)^2 sqrt(2 S:S) on the interior and the ghost
// layer (a ghost takes the value of its zero-gradient / periodic source).
// grid (ceil((nx+2)/64), ny+2, nz+2), block 64.
__global__ void les_nut_kernel(LDev q, const float *__restrict__ u, const float *__restrict__ v,
                               const float *__restrict__ w, float *__restrict__ nut)
{
    const PDims &d = q.d;
    const int gi = blockIdx.x * blockDim.x + threadIdx.x;
    const int gj = blockIdx.y, gk = blockIdx.z;
    if (gi > d.nx + 1) return;
    const int i = min(max(gi, 1), d.nx);
    const int j = gj == 0 ? d.ny : (gj == d.ny + 1 ? 1 : gj);
    const int k = min(max(gk, 1), d.nz);
    const float r = q.rdx;
    const float s11 = (u[L(d, i, j, k)] - u[L(d, i - 1, j, k)]) * r;
    const float s22 = (v[L(d, i, j, k)] - v[L(d, i, j - 1, k)]) * r;
    const float s33 = (w[L(d, i, j, k)] - w[L(d, i, j, k - 1)]) * r;
    float a12 = 0.0f, a13 = 0.0f, a23 = 0.0f;
#pragma unroll
    for (int a = -1; a <= 0; ++a)
#pragma unroll
        for (int b = -1; b <= 0; ++b) {
            const float e12 = s12e(d, r, u, v, i + a, j + b, k);
            const float e13 = s13e(d, r, u, w, i + a, j, k + b);
            const float e23 = s23e(d, r, v, w, i, j + a, k + b);
            a12 += e12 * e12;
            a13 += e13 * e13;
            a23 += e23 * e23;
        }
    const float ss = 2.0f * (s11 * s11 + s22 * s22 + s33 * s33) + (a12 + a13 + a23);
    nut[L(d, gi, gj, gk)] = q.l2 * sqrtf(ss);
}

// velfg + feedbf + viscous terms + adam on the three faces owned by cell
// (i,j,k): reads u^n (with ghosts) and nu_t, writes u* to the other buffer
// set and updates F_old and the Goldstein integrals in place.
// grid (ceil(nx/32), ceil(ny/4), nz), block (32, 4).
__global__ void __launch_bounds__(128)
les_predict_kernel(LDev q, int first, const float *__restrict__ u, const float *__restrict__ v,
                   const float *__restrict__ w, const float *__restrict__ nut, const uint8_t *__restrict__ face,
                   float *__restrict__ us, float *__restrict__ vs, float *__restrict__ ws, float *__restrict__ fuo,
                   float *__restrict__ fvo, float *__restrict__ fwo, float *__restrict__ gu, float *__restrict__ gv,
                   float *__restrict__ gw)
{
    const PDims &d = q.d;
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y * blockDim.y + threadIdx.y + 1;
    const int k = blockIdx.z + 1;
    if (i > d.nx || j > d.ny) return;
    const float r = q.rdx, nu = q.nu;
    const long long c = L(d, i, j, k);
    const long long sx = 1, sy = d.pitch, sz = d.plane;
    auto U = [&](long long o) { return u[c + o]; };
    auto V = [&](long long o) { return v[c + o]; };
    auto W = [&](long long o) { return w[c + o]; };
    auto NE = [&](long long o) { return nu + nut[c + o]; };
    // stresses at their natural points, offsets relative to cell c
    auto T11 = [&](long long o) { return 2.0f * NE(o) * (U(o) - U(o - sx)) * r; };
    auto T22 = [&](long long o) { return 2.0f * NE(o) * (V(o) - V(o - sy)) * r; };
    auto T33 = [&](long long o) { return 2.0f * NE(o) * (W(o) - W(o - sz)) * r; };
    auto T12 = [&](long long o) {  // xy edge east-north of cell c+o
        const float s = 0.5f * ((U(o + sy) - U(o)) + (V(o + sx) - V(o))) * r;
        const float ne = 0.25f * ((NE(o) + NE(o + sx)) + (NE(o + sy) + NE(o + sx + sy)));
        return 2.0f * ne * s;
    };
    auto T13 = [&](long long o) {  // xz edge east-top of cell c+o
        const float s = 0.5f * ((U(o + sz) - U(o)) + (W(o + sx) - W(o))) * r;
        const float ne = 0.25f * ((NE(o) + NE(o + sx)) + (NE(o + sz) + NE(o + sx + sz)));
        return 2.0f * ne * s;
    };
    auto T23 = [&](long long o) {  // yz edge north-top of cell c+o
        const float s = 0.5f * ((V(o + sz) - V(o)) + (W(o + sy) - W(o))) * r;
        const float ne = 0.25f * ((NE(o) + NE(o + sy)) + (NE(o + sz) + NE(o + sy + sz)));
        return 2.0f * ne * s;
    };
    const uint8_t fl = face[c];
    const float dt = q.dt;
    const float t12 = T12(0), t13 = T13(0), t23 = T23(0);

    // ---- u face (i+1/2, j, k)
    {
        const float ue = 0.5f * (U(0) + U(sx)), uw = 0.5f * (U(-sx) + U(0));
        const float un = 0.5f * (U(0) + U(sy)) * 0.5f * (V(0) + V(sx));
        const float us_ = 0.5f * (U(-sy) + U(0)) * 0.5f * (V(-sy) + V(sx - sy));
        const float ut = 0.5f * (U(0) + U(sz)) * 0.5f * (W(0) + W(sx));
        const float ub = 0.5f * (U(-sz) + U(0)) * 0.5f * (W(-sz) + W(sx - sz));
        float f = -r * ((ue * ue - uw * uw) + (un - us_) + (ut - ub));
        if (fl & FACE_U) {
            const float g = gu[c] + dt * U(0);
            gu[c] = g;
            f += q.alpha * g + q.beta * U(0);
        }
        f += r * ((T11(sx) - T11(0)) + (t12 - T12(-sy)) + (t13 - T13(-sz)));
        const float fo = fuo[c];
        us[c] = U(0) + dt * (first ? f : 1.5f * f - 0.5f * fo);
        fuo[c] = f;
    }
    // ---- v face (i, j+1/2, k)
    {
        const float ve = 0.5f * (V(0) + V(sx)) * 0.5f * (U(0) + U(sy));
        const float vw = 0.5f * (V(-sx) + V(0)) * 0.5f * (U(-sx) + U(sy - sx));
        const float vn = 0.5f * (V(0) + V(sy)), vs_ = 0.5f * (V(-sy) + V(0));
        const float vt = 0.5f * (V(0) + V(sz)) * 0.5f * (W(0) + W(sy));
        const float vb = 0.5f * (V(-sz) + V(0)) * 0.5f * (W(-sz) + W(sy - sz));
        float f = -r * ((ve - vw) + (vn * vn - vs_ * vs_) + (vt - vb));
        if (fl & FACE_V) {
            const float g = gv[c] + dt * V(0);
            gv[c] = g;
            f += q.alpha * g + q.beta * V(0);
        }
        f += r * ((t12 - T12(-sx)) + (T22(sy) - T22(0)) + (t23 - T23(-sz)));
        const float fo = fvo[c];
        vs[c] = V(0) + dt * (first ? f : 1.5f * f - 0.5f * fo);
        fvo[c] = f;
    }
    // ---- w face (i, j, k+1/2)
    if (k < d.nz) {
        const float we = 0.5f * (W(0) + W(sx)) * 0.5f * (U(0) + U(sz));
        const float ww = 0.5f * (W(-sx) + W(0)) * 0.5f * (U(-sx) + U(sz - sx));
        const float wn = 0.5f * (W(0) + W(sy)) * 0.5f * (V(0) + V(sz));
        const float ws_ = 0.5f * (W(-sy) + W(0)) * 0.5f * (V(-sy) + V(sz - sy));
        const float wt = 0.5f * (W(0) + W(sz)), wb = 0.5f * (W(-sz) + W(0));
        float f = -r * ((we - ww) + (wn - ws_) + (wt * wt - wb * wb));
        if (fl & FACE_W) {
            const float g = gw[c] + dt * W(0);
            gw[c] = g;
            f += q.alpha * g + q.beta * W(0);
        }
        f += r * ((t13 - T13(-sx)) + (t23 - T23(-sy)) + (T33(sz) - T33(0)));
        const float fo = fwo[c];
        ws[c] = W(0) + dt * (first ? f : 1.5f * f - 0.5f * fo);
        fwo[c] = f;
    }
    if (i == 1) us[c - 1] = U(-sx);  // the inflow face travels with u*
}

// b = div(u*) / dt at interior cells.
__global__ void les_rhs_kernel(LDev q, const float *__restrict__ u, const float *__restrict__ v,
                               const float *__restrict__ w, float *__restrict__ b)
{
    const PDims &d = q.d;
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y + 1, k = blockIdx.z + 1;
    if (i > d.nx) return;
    const long long c = L(d, i, j, k);
    const float vs = v[L(d, i, (j > 1) ? j - 1 : d.ny, k)];
    b[c] = q.rdxdt * ((u[c] - u[c - 1]) + (v[c] - vs) + (w[c] - w[c - d.plane]));
}

}  // namespace

struct gbsw_les {
    gbsw_les_params p;
    LDev q;
    cudaStream_t stream;
    float *U[2], *V[2], *W[2];  // [cur] holds u* between steps
    int cur;
    float *fuo, *fvo, *fwo, *gu, *gv, *gw, *nut, *b, *uin;
    uint8_t *face;
    PoissonSolver solver;
    PoissonCtl *ctl_log;   // per-step copies of the solver control block
    int ctl_log_len;
    int step;
    int fixed_iters;       // > 0: paper mode, exactly this many SOR iterations per step
    gbsw_unet *net;        // learned warm start (not owned), NULL = previous pressure
    int ws_factor;         // the network runs on the grid coarsened by this factor (0 = default)
    double *ws_scratch;    // restriction passes of the warm start
    size_t ws_scratch_n;
    size_t n;              // elements per padded field
};

namespace {

// True if the network fits the grid coarsened by f.
bool ws_fits(const gbsw_les *s, int f)
{
    const int nx = s->q.d.nx, ny = s->q.d.ny, nz = s->q.d.nz;
    return ws_factor_ok(nx, ny, nz, f) && unet_shape_ok(nz / f, ny / f, nx / f);
}

// Coarsening factor of the learned warm start: the one set, else the
// largest power of two <= 16 at which the network fits the coarse grid.
int ws_factor_of(const gbsw_les *s)
{
    if (s->ws_factor > 0) return s->ws_factor;
    for (int f = 16; f > 1; f >>= 1)
        if (ws_fits(s, f)) return f;
    return 1;
}

gbsw_status les_alloc(gbsw_les *s)
{
    const size_t fb = s->n * sizeof(float);
    float **fl[] = {&s->U[0], &s->U[1], &s->V[0], &s->V[1], &s->W[0], &s->W[1], &s->fuo, &s->fvo, &s->fwo,
                    &s->gu, &s->gv, &s->gw, &s->nut, &s->b};
    for (float **pp : fl) {
        GBSW_CUDA_TRY(cudaMalloc((void **)pp, fb));
        GBSW_CUDA_TRY(cudaMemsetAsync(*pp, 0, fb, s->stream));
    }
    GBSW_CUDA_TRY(cudaMalloc((void **)&s->uin, (size_t)(s->p.nz + 2) * sizeof(float)));
    GBSW_CUDA_TRY(cudaMalloc((void **)&s->face, s->n));
    GBSW_CUDA_TRY(cudaMemsetAsync(s->face, 0, s->n, s->stream));
    return GBSW_OK;
}

double inflow_profile(const gbsw_les_params &P, int k)
{
    const double z = ((double)k - 0.5) * P.dx;
    return P.u_ref * log(z / P.z0) / log(P.z_ref / P.z0);
}

gbsw_status ensure_ctl_log(gbsw_les *s, int n)
{
    if (n <= s->ctl_log_len) return GBSW_OK;
    if (s->ctl_log) cudaFree(s->ctl_log);
    s->ctl_log = nullptr;
    s->ctl_log_len = 0;
    GBSW_CUDA_TRY(cudaMalloc((void **)&s->ctl_log, (size_t)n * sizeof(PoissonCtl)));
    s->ctl_log_len = n;
    return GBSW_OK;
}

// Enqueue the predictor part of one step (velnw ... rhs).
gbsw_status les_predictor(gbsw_les *s)
{
    const LDev &q = s->q;
    const PDims &d = q.d;
    const int a = s->cur, bset = 1 - s->cur;
    float *u = s->U[a], *v = s->V[a], *w = s->W[a];
    const dim3 g1(ceil_div(d.nx, 128), d.ny, d.nz), b1(128);
    les_velnw_kernel<<<g1, b1, 0, s->stream>>>(q, s->solver.p_hi, u, v, w);
    les_bc_x_kernel<<<dim3(ceil_div(d.ny, 128), d.nz), 128, 0, s->stream>>>(q, s->uin, u, v, w);
    les_bc_y_kernel<<<dim3(ceil_div(d.nx + 2, 128), d.nz), 128, 0, s->stream>>>(q, u, v, w);
    les_bc_z_kernel<<<dim3(ceil_div(d.nx + 2, 128), d.ny + 2), 128, 0, s->stream>>>(q, u, v, w);
    les_nut_kernel<<<dim3(ceil_div(d.nx + 2, 64), d.ny + 2, d.nz + 2), 64, 0, s->stream>>>(q, u, v, w, s->nut);
    les_predict_kernel<<<dim3(ceil_div(d.nx, 32), ceil_div(d.ny, 4), d.nz), dim3(32, 4), 0, s->stream>>>(
        q, s->step == 0, u, v, w, s->nut, s->face, s->U[bset], s->V[bset], s->W[bset], s->fuo, s->fvo, s->fwo,
        s->gu, s->gv, s->gw);
    les_rhs_kernel<<<g1, b1, 0, s->stream>>>(q, s->U[bset], s->V[bset], s->W[bset], s->b);
    GBSW_LAUNCH_CHECK();
    s->cur = bset;
    return GBSW_OK;
}

float *field_f32(gbsw_les *s, int id)
{
    switch (id) {
    case GBSW_LES_U: return s->U[s->cur];
    case GBSW_LES_V: return s->V[s->cur];
    case GBSW_LES_W: return s->W[s->cur];
    case GBSW_LES_FU_OLD: return s->fuo;
    case GBSW_LES_FV_OLD: return s->fvo;
    case GBSW_LES_FW_OLD: return s->fwo;
    case GBSW_LES_GU: return s->gu;
    case GBSW_LES_GV: return s->gv;
    case GBSW_LES_GW: return s->gw;
    case GBSW_LES_NUT: return s->nut;
    case GBSW_LES_B: return s->b;
    default: return nullptr;
    }
}

}  // namespace

extern "C" {

gbsw_status les_create(const gbsw_les_params *params, const uint8_t *solid, void *stream, gbsw_les **out)
{
    if (!params || !out) return GBSW_ERR_ARG;
    const gbsw_les_params P = *params;
    if (P.nx < 2 || P.ny < 2 || P.nz < 2 || (P.ny & 1) || P.nx > 4096 || P.ny > 4096 || P.nz > 4096) return GBSW_ERR_ARG;
    if (!(P.dx > 0) || !(P.dt > 0) || !(P.z0 > 0) || !(P.z_ref > P.z0) || !(P.cs >= 0) || !(P.nu >= 0) ||
        !(P.omega > 0 && P.omega < 2) || !(P.tol >= 0) || P.max_iter < 0 || P.check_every < 1 || P.check_every > 1000)
        return GBSW_ERR_ARG;
    if (0.5 * P.dx <= P.z0) return GBSW_ERR_ARG;
    if (fault_injected("alloc")) return GBSW_ERR_OOM;
    // advective CFL of the fastest inflow speed
    double umax = 0.0;
    for (int k = 1; k <= P.nz; ++k) umax = std::max(umax, fabs(inflow_profile(P, k)));
    if (umax * P.dt / P.dx > 0.5) return GBSW_ERR_CFL;

    gbsw_les *s = new (std::nothrow) gbsw_les();
    if (!s) return GBSW_ERR_OOM;
    s->p = P;
    s->stream = (cudaStream_t)stream;
    s->cur = 0;
    s->step = 0;
    gbsw_status st = s->solver.init(P.nx, P.ny, P.nz, P.dx, nullptr, s->stream);
    if (st == GBSW_OK) st = s->solver.configure(P.omega, P.tol, P.max_iter, P.check_every);
    LDev &q = s->q;
    q.d = s->solver.d;
    q.dt = (float)P.dt;
    q.rdx = (float)(1.0 / P.dx);
    q.c_grad = (float)(P.dt / P.dx);
    q.l2 = (float)((P.cs * P.dx) * (P.cs * P.dx));
    q.nu = (float)P.nu;
    q.alpha = (float)P.alpha;
    q.beta = (float)P.beta;
    q.rdxdt = (float)(1.0 / (P.dx * P.dt));
    s->n = (size_t)q.d.plane * (size_t)(P.nz + 2);
    if (st == GBSW_OK) st = les_alloc(s);
    if (st != GBSW_OK) {
        les_destroy(s);
        return st;
    }
    s->solver.b = s->b;

    // face flags and the initial u* (inflow profile on open x-faces)
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int pitch = q.d.pitch;
    const long long plane = q.d.plane;
    std::vector<uint8_t> face(s->n, 0);
    std::vector<float> u0(s->n, 0.0f), uin(nz + 2, 0.0f);
    auto S = [&](int i, int j, int k) -> int {
        if (!solid || i < 1 || i > nx || k < 1 || k > nz) return 0;
        if (j < 1) j += ny;
        if (j > ny) j -= ny;
        return solid[((size_t)(k - 1) * ny + (j - 1)) * nx + (i - 1)] != 0;
    };
    for (int k = 1; k <= nz; ++k) uin[k] = (float)inflow_profile(P, k);
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                const size_t c = (size_t)k * plane + (size_t)j * pitch + i;
                const int sc = S(i, j, k);
                uint8_t f = 0;
                if (sc || S(i + 1, j, k)) f |= FACE_U;
                if (i >= 1 && (sc || S(i, j + 1, k))) f |= FACE_V;
                if (i >= 1 && k < nz && (sc || S(i, j, k + 1))) f |= FACE_W;
                if (i >= 1) face[c] = f;
                u0[c] = (f & FACE_U) ? 0.0f : uin[k];
            }
    cudaError_t e = cudaMemcpyAsync(s->face, face.data(), s->n, cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->U[0], u0.data(), s->n * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->uin, uin.data(), (nz + 2) * sizeof(float), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
        record_cuda_error(e, "les_create upload", __FILE__, __LINE__);
        les_destroy(s);
        return GBSW_ERR_CUDA;
    }
    *out = s;
    return GBSW_OK;
}

gbsw_status les_step(gbsw_les *s, int nsteps, gbsw_les_stats *stats)
{
    gbsw::NvtxRange nvtx_range("les_step");
    if (!s || nsteps < 0) return GBSW_ERR_ARG;
    if (nsteps == 0) return GBSW_OK;
    gbsw_status st = ensure_ctl_log(s, nsteps);
    if (st != GBSW_OK) return st;
    std::vector<cudaEvent_t> ev;
    if (stats) {
        ev.resize(4 * (size_t)nsteps);
        for (auto &x : ev) GBSW_CUDA_TRY(cudaEventCreate(&x));
    }
    PadDims pd;
    pd.nx = s->q.d.nx;
    pd.ny = s->q.d.ny;
    pd.nz = s->q.d.nz;
    pd.pitch = s->q.d.pitch;
    pd.plane = s->q.d.plane;
    for (int t = 0; t < nsteps && st == GBSW_OK; ++t) {
        if (stats) cudaEventRecord(ev[4 * t], s->stream);
        st = les_predictor(s);
        if (st != GBSW_OK) break;
        if (stats) cudaEventRecord(ev[4 * t + 1], s->stream);
        if (s->net) {
            const int f = ws_factor_of(s);
            const size_t need = ws_scratch_doubles(pd.nx, pd.ny, pd.nz, f);
            if (need > s->ws_scratch_n) {
                cudaStreamSynchronize(s->stream);
                cudaFree(s->ws_scratch);
                s->ws_scratch_n = 0;
                if (cudaMalloc((void **)&s->ws_scratch, need * sizeof(double)) != cudaSuccess) {
                    s->ws_scratch = nullptr;
                    st = GBSW_ERR_OOM;
                    break;
                }
                s->ws_scratch_n = need;
            }
            st = unet_warm_start(s->net, s->b, s->solver.p_hi, pd, s->p.dx, f, s->ws_scratch, s->stream);
            if (st != GBSW_OK) break;
        }
        if (stats) cudaEventRecord(ev[4 * t + 2], s->stream);
        st = s->fixed_iters > 0 ? s->solver.enqueue_fixed(s->fixed_iters, true) : s->solver.enqueue();
        if (st != GBSW_OK) break;
        if (stats) cudaEventRecord(ev[4 * t + 3], s->stream);
        st = s->solver.record(s->ctl_log + t);
        s->step += 1;
    }
    std::vector<PoissonCtl> log(nsteps);
    cudaError_t e = cudaMemcpyAsync(log.data(), s->ctl_log, nsteps * sizeof(PoissonCtl), cudaMemcpyDeviceToHost,
                                    s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess && st == GBSW_OK) {
        record_cuda_error(e, "les_step", __FILE__, __LINE__);
        st = GBSW_ERR_CUDA;
    }
    gbsw_status worst = GBSW_OK;
    for (int t = 0; t < nsteps && st == GBSW_OK; ++t) {
        const PoissonCtl &c = log[t];
        gbsw_status one = GBSW_OK;
        if (c.status != DEV_OK) one = dev_status_to_gbsw(c.status);
        else if (s->fixed_iters == 0 && !(c.rho <= s->p.tol || c.bb < 1e-60)) one = GBSW_NOT_CONVERGED;
        if (stats) {
            stats[t].iters = c.iters;
            stats[t].status = one;
            stats[t].rel_res = c.rho;
            cudaEventElapsedTime(&stats[t].ms_predictor, ev[4 * t], ev[4 * t + 1]);
            cudaEventElapsedTime(&stats[t].ms_guess, ev[4 * t + 1], ev[4 * t + 2]);
            cudaEventElapsedTime(&stats[t].ms_solve, ev[4 * t + 2], ev[4 * t + 3]);
        }
        if (one < 0 && worst >= 0) worst = one;
        else if (one == GBSW_NOT_CONVERGED && worst == GBSW_OK) worst = one;
    }
    for (auto &x : ev) cudaEventDestroy(x);
    return st != GBSW_OK ? st : worst;
}

gbsw_status les_get_field(gbsw_les *s, int field, void *host)
{
    if (!s || !host) return GBSW_ERR_ARG;
    const PDims &d = s->q.d;
    const size_t rows = (size_t)(d.ny + 2) * (size_t)(d.nz + 2);
    if (field == GBSW_LES_P) {
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(host, (d.nx + 2) * sizeof(double), s->solver.p_hi, d.pitch * sizeof(double),
                                        (d.nx + 2) * sizeof(double), rows, cudaMemcpyDeviceToHost, s->stream));
    } else {
        float *src = field_f32(s, field);
        if (!src) return GBSW_ERR_ARG;
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(host, (d.nx + 2) * sizeof(float), src, d.pitch * sizeof(float),
                                        (d.nx + 2) * sizeof(float), rows, cudaMemcpyDeviceToHost, s->stream));
    }
    GBSW_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return GBSW_OK;
}

gbsw_status les_set_field(gbsw_les *s, int field, const void *host)
{
    if (!s || !host) return GBSW_ERR_ARG;
    const PDims &d = s->q.d;
    const size_t rows = (size_t)(d.ny + 2) * (size_t)(d.nz + 2);
    if (field == GBSW_LES_P) {
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(s->solver.p_hi, d.pitch * sizeof(double), host, (d.nx + 2) * sizeof(double),
                                        (d.nx + 2) * sizeof(double), rows, cudaMemcpyHostToDevice, s->stream));
    } else {
        float *dst = field_f32(s, field);
        if (!dst) return GBSW_ERR_ARG;
        GBSW_CUDA_TRY(cudaMemcpy2DAsync(dst, d.pitch * sizeof(float), host, (d.nx + 2) * sizeof(float),
                                        (d.nx + 2) * sizeof(float), rows, cudaMemcpyHostToDevice, s->stream));
    }
    GBSW_CUDA_TRY(cudaStreamSynchronize(s->stream));
    return GBSW_OK;
}

gbsw_status les_get_state(gbsw_les *s, gbsw_les_state *st)
{
    if (!s || !st) return GBSW_ERR_ARG;
    void *bufs[10] = {st->u, st->v, st->w, st->p, st->fu_old, st->fv_old, st->fw_old, st->gu, st->gv, st->gw};
    for (int f = 0; f < 10; ++f)
        if (bufs[f]) {
            gbsw_status r = les_get_field(s, f, bufs[f]);
            if (r != GBSW_OK) return r;
        }
    st->step = s->step;
    return GBSW_OK;
}

gbsw_status les_set_state(gbsw_les *s, const gbsw_les_state *st)
{
    if (!s || !st || st->step < 0) return GBSW_ERR_ARG;
    const void *bufs[10] = {st->u, st->v, st->w, st->p, st->fu_old, st->fv_old, st->fw_old, st->gu, st->gv, st->gw};
    for (int f = 0; f < 10; ++f)
        if (bufs[f]) {
            gbsw_status r = les_set_field(s, f, bufs[f]);
            if (r != GBSW_OK) return r;
        }
    s->step = st->step;
    return GBSW_OK;
}

gbsw_status les_get_step(gbsw_les *s, int *step)
{
    if (!s || !step) return GBSW_ERR_ARG;
    *step = s->step;
    return GBSW_OK;
}

gbsw_status les_set_step(gbsw_les *s, int step)
{
    if (!s || step < 0) return GBSW_ERR_ARG;
    s->step = step;
    return GBSW_OK;
}

gbsw_status les_set_warm_start(gbsw_les *s, gbsw_unet *net)
{
    if (!s) return GBSW_ERR_ARG;
    if (net && !ws_fits(s, ws_factor_of(s))) return GBSW_ERR_ARG;
    s->net = net;
    return GBSW_OK;
}

gbsw_status les_set_warm_start_factor(gbsw_les *s, int f)
{
    if (!s || f < 0 || (f != 0 && !ws_fits(s, f))) return GBSW_ERR_ARG;
    s->ws_factor = f;
    return GBSW_OK;
}

gbsw_status les_set_fixed_iterations(gbsw_les *s, int niter)
{
    if (!s || niter < 0) return GBSW_ERR_ARG;
    s->fixed_iters = niter;
    return GBSW_OK;
}

gbsw_status les_set_solver(gbsw_les *s, double omega, double tol, int max_iter, int check_every)
{
    if (!s) return GBSW_ERR_ARG;
    gbsw_status st = s->solver.configure(omega, tol, max_iter, check_every);
    if (st == GBSW_OK) {
        s->p.omega = omega;
        s->p.tol = tol;
        s->p.max_iter = max_iter;
        s->p.check_every = check_every;
    }
    return st;
}

void les_destroy(gbsw_les *s)
{
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    for (int b = 0; b < 2; ++b) {
        cudaFree(s->U[b]);
        cudaFree(s->V[b]);
        cudaFree(s->W[b]);
    }
    float *fl[] = {s->fuo, s->fvo, s->fwo, s->gu, s->gv, s->gw, s->nut, s->b, s->uin};
    for (float *x : fl) cudaFree(x);
    cudaFree(s->face);
    cudaFree(s->ctl_log);
    cudaFree(s->ws_scratch);
    s->solver.release();
    delete s;
}

}  // extern "C"

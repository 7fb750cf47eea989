// UFLES time step (Sec. 6.3.1 of arXiv:1711.04471): velnw -> bondv1 ->
// velfg -> feedbf -> les -> adam -> press, on the GPU.
//
// Kernels per step:
//   les_velnw_kernel         u = u* - dt grad p                  (velnw)
//   les_predict_tile_kernel  ghost layer + Smagorinsky nu_t +
//                            advection + Goldstein forcing + viscous
//                            stress divergence + Adams-Bashforth (bondv1, les, velfg, feedbf, adam)
//   les_rhs_kernel           b = div(u*) / dt                    (press, right-hand side)
//   PoissonSolver            red-black SOR to the FP64 tolerance (press)
// The paper's compiler emitted 29 map and 4 reduction kernels for this
// loop; here everything between velnw and the right-hand side is one
// kernel.  velnw stays apart: its pressure differences are FP64, which
// runs at a small fraction of the FP32 rate on this GPU, and a fused tile
// would recompute them on every halo cell.
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

namespace gbsw {

// Out-of-range index count of the bounds-checked debug build.
static __device__ unsigned g_les_bounds;

unsigned long long take_bounds_les()
{
    unsigned h = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&h, g_les_bounds, sizeof(h)) != cudaSuccess) return 0;
    cudaMemcpyToSymbol(g_les_bounds, &zero, sizeof(zero));
    return h;
}

}  // namespace gbsw

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

// Index test of the bounds-checked build: c inside a padded field
// ((nz+2) planes); always true in the product build.
#define LES_OK(d, c) GBSW_INBOUNDS((c), (long long)(d).plane * ((d).nz + 2), &g_les_bounds)

// velnw: projection with the previous pressure, interior faces only.
__global__ void les_velnw_kernel(LDev q, const double *__restrict__ p, float *__restrict__ u, float *__restrict__ v,
                                 float *__restrict__ w)
{
    const PDims &d = q.d;
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y + 1, k = blockIdx.z + 1;
    if (i > d.nx) return;
    const long long c = L(d, i, j, k), cn = L(d, i, (j < d.ny) ? j + 1 : 1, k);
    if (!LES_OK(d, c) || !LES_OK(d, c + 1) || !LES_OK(d, cn) || !LES_OK(d, c + d.plane)) return;
    const double pc = p[c];
    const double pe = (i < d.nx) ? p[c + 1] : -pc;
    const double pn = p[cn];
    u[c] -= q.c_grad * (float)(pe - pc);
    v[c] -= q.c_grad * (float)(pn - pc);
    if (k < d.nz) w[c] -= q.c_grad * (float)(p[c + d.plane] - pc);
}

// ---------------------------------------------------------------- fused predictor
// bondv1 + les (nu_t) + velfg + feedbf + viscous terms + adam in one pass.
// A CTA owns LT_X x LT_Y columns of cells and marches up a chunk of LT_KZ
// planes.  Shared memory holds a ring of LT_US planes of u, v, w (after
// velnw) with a 2-cell halo in x and y, and a ring of LT_ES planes of nu_t
// with a 1-cell halo; each plane step loads plane k+2, forms nu_t on plane
// k+1 and predicts plane k, with two barriers.  The ghost layer of bondv1
// is formed while loading (never stored): inflow profile and reflected v, w
// at i = 0, zero gradient at i = nx+1, periodic rows, no slip at the ground,
// free slip at the lid, w = 0 on the ground and lid faces; a ghost nu_t is
// that of its zero-gradient / periodic source.  The arithmetic of every
// term is that of the oracle's subroutines (Sec. 6.3.1).
constexpr int LT_X = 32, LT_Y = 8, LT_THREADS = LT_X * LT_Y;
constexpr int LT_HX = LT_X + 4, LT_HY = LT_Y + 4, LT_HN = LT_HX * LT_HY;  // velocity planes, halo 2
constexpr int LT_EX = LT_X + 2, LT_EY = LT_Y + 2, LT_EN = LT_EX * LT_EY;  // nu_t planes, halo 1
constexpr int LT_US = 5, LT_ES = 3;  // ring slots: planes k-2 .. k+2 and k-1 .. k+1 of plane step k
constexpr int LT_KZ = 8;             // planes per CTA (8 and 16 tie on large grids; 8 keeps small grids parallel)

struct LesTileSmem {
    float vel[LT_US][3][LT_HN];  // u, v, w
    float nut[LT_ES][LT_EN];
};

__device__ __forceinline__ int lt_uslot(int k) { return (k + LT_US) % LT_US; }
__device__ __forceinline__ int lt_eslot(int k) { return (k + LT_ES) % LT_ES; }

constexpr int LT_LPT = (LT_HN + LT_THREADS - 1) / LT_THREADS;  // velocity cells a thread loads per plane
constexpr int LT_NPT = (LT_EN + LT_THREADS - 1) / LT_THREADS;  // nu_t cells a thread forms per plane

// The cells a thread loads of every velocity plane and forms of every nu_t
// plane, fixed for the whole march (so no plane step repeats the index
// arithmetic).
struct LtMap {
    int src[LT_LPT];   // in-plane offset of the loaded cell's source (row wrapped, column clamped); -1: zero
    unsigned inflow;   // bit c: loaded cell c is on the inflow face i = 0
    int o[LT_NPT];     // velocity-plane offset of nu_t cell c's source (column clamped); -1: not formed
    int out[LT_NPT];   // in-plane offset of nu_t cell c in the output field; -1: not this CTA's cell
};

__device__ __forceinline__ LtMap lt_map(const PDims &d, int i0, int j0)
{
    LtMap m;
    m.inflow = 0;
#pragma unroll
    for (int c = 0; c < LT_LPT; ++c) {
        const int idx = threadIdx.x + c * LT_THREADS;
        const int lx = idx % LT_HX, ly = idx / LT_HX;
        const int i = i0 - 1 + lx, j = j0 - 1 + ly;
        m.src[c] = -1;
        if (idx < LT_HN && i >= 0 && i <= d.nx + 1) {  // columns outside the ghost layer are never read
            int jw = (j - 1) % d.ny;
            if (jw < 0) jw += d.ny;
            jw += 1;  // periodic rows
            const int ic = i == 0 ? 1 : (i == d.nx + 1 ? d.nx : i);
            m.src[c] = jw * d.pitch + ic;
            if (i == 0) m.inflow |= 1u << c;
        }
    }
#pragma unroll
    for (int c = 0; c < LT_NPT; ++c) {
        const int idx = threadIdx.x + c * LT_THREADS;
        const int ex = idx % LT_EX, ey = idx / LT_EX;
        const int i = i0 + ex, j = j0 + ey;
        m.o[c] = -1;
        m.out[c] = -1;
        if (idx < LT_EN && i <= d.nx + 1) {  // past the ghost column: never read
            const int ic = min(max(i, 1), d.nx);
            m.o[c] = (ey + 1) * LT_HX + (ic - i0 + 1);
            if (ex >= 1 && ex <= LT_X && ey >= 1 && ey <= LT_Y && i <= d.nx && j <= d.ny) m.out[c] = j * d.pitch + i;
        }
    }
    return m;
}

struct LtVel {
    float u[LT_LPT], v[LT_LPT], w[LT_LPT];
};

// Global reads of velocity plane kk after bondv1, into registers (zeros
// for a plane outside 0 .. nz+1, which no stage reads): ground ghost
// reflected u, v; lid ghost copied u, v; w = 0 on both and on the lid
// face; inflow profile and reflected v, w at i = 0.
__device__ __forceinline__ LtVel lt_fetch_plane(const LDev &q, const LtMap &m, int kk, const float *__restrict__ u,
                                                const float *__restrict__ v, const float *__restrict__ w,
                                                const float *__restrict__ uin)
{
    const PDims &d = q.d;
    LtVel r;
    const bool ok = kk >= 0 && kk <= d.nz + 1;
    const int kc = kk <= 0 ? 1 : (kk >= d.nz + 1 ? d.nz : kk);
    const bool ground = kk == 0, wzero = kk == 0 || kk >= d.nz;
    const long long base = (long long)kc * d.plane;
    const float uin_k = ok && GBSW_INBOUNDS(kc, d.nz + 2, &g_les_bounds) ? uin[kc] : 0.0f;
#pragma unroll
    for (int c = 0; c < LT_LPT; ++c) {
        float a = 0.0f, b = 0.0f, cw = 0.0f;
        if (ok && m.src[c] >= 0 && LES_OK(d, base + m.src[c])) {
            const long long cc = base + m.src[c];
            const bool in = (m.inflow >> c) & 1u;
            const float uu = in ? uin_k : u[cc];
            float vv = v[cc], ww = w[cc];
            if (in) {
                vv = -vv;
                ww = -ww;
            }
            a = ground ? -uu : uu;
            b = ground ? -vv : vv;
            cw = wzero ? 0.0f : ww;
        }
        r.u[c] = a;
        r.v[c] = b;
        r.w[c] = cw;
    }
    return r;
}

__device__ __forceinline__ void lt_store_plane(LesTileSmem &sm, const LtVel &r, int kk)
{
    float *pu = sm.vel[lt_uslot(kk)][0], *pv = sm.vel[lt_uslot(kk)][1], *pw = sm.vel[lt_uslot(kk)][2];
#pragma unroll
    for (int c = 0; c < LT_LPT; ++c) {
        const int idx = threadIdx.x + c * LT_THREADS;
        if (idx >= LT_HN) continue;
        pu[idx] = r.u[c];
        pv[idx] = r.v[c];
        pw[idx] = r.w[c];
    }
}

// nu_t = (cs dx)^2 sqrt(2 S:S) on plane kk (0 .. nz+1) of the tile and its
// 1-cell halo, from velocity planes kc-1 .. kc+1 (kc = kk clamped to
// 1 .. nz; a ghost column takes the value of i clamped to 1 .. nx; rows
// are periodic through the loaded planes).  The CTA's own interior cells
// are also written to nut_out when write is set.
__device__ __forceinline__ void lt_nut_plane(const LDev &q, LesTileSmem &sm, const LtMap &m, int kk, bool write,
                                             float *__restrict__ nut_out)
{
    const PDims &d = q.d;
    if (kk < 0 || kk > d.nz + 1) return;
    const int kc = min(max(kk, 1), d.nz);
    const float *um = sm.vel[lt_uslot(kc - 1)][0], *uc = sm.vel[lt_uslot(kc)][0], *up = sm.vel[lt_uslot(kc + 1)][0];
    const float *vm = sm.vel[lt_uslot(kc - 1)][1], *vc = sm.vel[lt_uslot(kc)][1], *vp = sm.vel[lt_uslot(kc + 1)][1];
    const float *wm = sm.vel[lt_uslot(kc - 1)][2], *wc = sm.vel[lt_uslot(kc)][2];
    float *ne = sm.nut[lt_eslot(kk)];
    const float r = q.rdx;
    const long long base = (long long)kk * d.plane;
#pragma unroll
    for (int c = 0; c < LT_NPT; ++c) {
        const int o = m.o[c];
        if (o < 0) continue;
        // velocity of cell (ic+a, j+b) on plane kc, kc-1 (m) or kc+1 (p)
        auto U = [&](int a, int b) { return uc[o + b * LT_HX + a]; };
        auto V = [&](int a, int b) { return vc[o + b * LT_HX + a]; };
        auto W = [&](int a, int b) { return wc[o + b * LT_HX + a]; };
        const float s11 = (U(0, 0) - U(-1, 0)) * r;
        const float s22 = (V(0, 0) - V(0, -1)) * r;
        const float s33 = (W(0, 0) - wm[o]) * r;
        float a12 = 0.0f, a13 = 0.0f, a23 = 0.0f;
#pragma unroll
        for (int a = -1; a <= 0; ++a)
#pragma unroll
            for (int b = -1; b <= 0; ++b) {
                // edges: xy at (ic+a, j+b, kc), xz at (ic+a, j, kc+b), yz at (ic, j+a, kc+b)
                const float *uz0 = b < 0 ? um : uc, *uz1 = b < 0 ? uc : up;
                const float *wz0 = b < 0 ? wm : wc;
                const float *vz0 = b < 0 ? vm : vc, *vz1 = b < 0 ? vc : vp;
                const float e12 = 0.5f * ((U(a, b + 1) - U(a, b)) + (V(a + 1, b) - V(a, b))) * r;
                const float e13 = 0.5f * ((uz1[o + a] - uz0[o + a]) + (wz0[o + a + 1] - wz0[o + a])) * r;
                const float e23 = 0.5f * ((vz1[o + a * LT_HX] - vz0[o + a * LT_HX]) +
                                          (wz0[o + (a + 1) * LT_HX] - wz0[o + a * LT_HX])) * r;
                a12 += e12 * e12;
                a13 += e13 * e13;
                a23 += e23 * e23;
            }
        const float ss = 2.0f * (s11 * s11 + s22 * s22 + s33 * s33) + (a12 + a13 + a23);
        const float nt = q.l2 * sqrtf(ss);
        ne[threadIdx.x + c * LT_THREADS] = nt;
        if (write && m.out[c] >= 0 && LES_OK(d, base + m.out[c])) nut_out[base + m.out[c]] = nt;
    }
}

// velfg + feedbf + viscous terms + adam on the three faces owned by the
// thread's cell (i, j, k) of plane k, from the velocity and nu_t rings.
// fl, fuo_c, fvo_c, fwo_c: the cell's face flags and F_old, read by the
// caller before the plane step's barriers (their latency hides behind the
// load and nu_t stages).
__device__ __forceinline__ void lt_predict_cell(const LDev &q, const LesTileSmem &sm, int k, int i, int j, int o,
                                                int on, bool first, uint8_t fl, float fuo_c, float fvo_c,
                                                float fwo_c, float *__restrict__ us, float *__restrict__ vs,
                                                float *__restrict__ ws, float *__restrict__ fuo,
                                                float *__restrict__ fvo, float *__restrict__ fwo,
                                                float *__restrict__ gu, float *__restrict__ gv, float *__restrict__ gw)
{
    const PDims &d = q.d;
    const float r = q.rdx, nu = q.nu;
    const float *vel[3] = {sm.vel[lt_uslot(k - 1)][0], sm.vel[lt_uslot(k)][0], sm.vel[lt_uslot(k + 1)][0]};
    const float *nut[3] = {sm.nut[lt_eslot(k - 1)], sm.nut[lt_eslot(k)], sm.nut[lt_eslot(k + 1)]};
    // value at cell (i+x, j+y, k+z), |x|, |y|, |z| <= 1 (field 0 u, 1 v, 2 w)
    auto F = [&](int f, int x, int y, int z) { return vel[z + 1][f * LT_HN + o + y * LT_HX + x]; };
    auto U = [&](int x, int y, int z) { return F(0, x, y, z); };
    auto V = [&](int x, int y, int z) { return F(1, x, y, z); };
    auto W = [&](int x, int y, int z) { return F(2, x, y, z); };
    auto NE = [&](int x, int y, int z) { return nu + nut[z + 1][on + y * LT_EX + x]; };
    // stresses at their natural points, offsets relative to the cell
    auto T11 = [&](int x, int y, int z) { return 2.0f * NE(x, y, z) * (U(x, y, z) - U(x - 1, y, z)) * r; };
    auto T22 = [&](int x, int y, int z) { return 2.0f * NE(x, y, z) * (V(x, y, z) - V(x, y - 1, z)) * r; };
    auto T33 = [&](int x, int y, int z) { return 2.0f * NE(x, y, z) * (W(x, y, z) - W(x, y, z - 1)) * r; };
    auto T12 = [&](int x, int y, int z) {  // xy edge east-north of cell (x, y, z)
        const float s = 0.5f * ((U(x, y + 1, z) - U(x, y, z)) + (V(x + 1, y, z) - V(x, y, z))) * r;
        const float ne = 0.25f * ((NE(x, y, z) + NE(x + 1, y, z)) + (NE(x, y + 1, z) + NE(x + 1, y + 1, z)));
        return 2.0f * ne * s;
    };
    auto T13 = [&](int x, int y, int z) {  // xz edge east-top
        const float s = 0.5f * ((U(x, y, z + 1) - U(x, y, z)) + (W(x + 1, y, z) - W(x, y, z))) * r;
        const float ne = 0.25f * ((NE(x, y, z) + NE(x + 1, y, z)) + (NE(x, y, z + 1) + NE(x + 1, y, z + 1)));
        return 2.0f * ne * s;
    };
    auto T23 = [&](int x, int y, int z) {  // yz edge north-top
        const float s = 0.5f * ((V(x, y, z + 1) - V(x, y, z)) + (W(x, y + 1, z) - W(x, y, z))) * r;
        const float ne = 0.25f * ((NE(x, y, z) + NE(x, y + 1, z)) + (NE(x, y, z + 1) + NE(x, y + 1, z + 1)));
        return 2.0f * ne * s;
    };
    const long long c = L(d, i, j, k);
    const float dt = q.dt;
    const float t12 = T12(0, 0, 0), t13 = T13(0, 0, 0), t23 = T23(0, 0, 0);
    // ---- u face (i+1/2, j, k)
    {
        const float ue = 0.5f * (U(0, 0, 0) + U(1, 0, 0)), uw = 0.5f * (U(-1, 0, 0) + U(0, 0, 0));
        const float un = 0.5f * (U(0, 0, 0) + U(0, 1, 0)) * 0.5f * (V(0, 0, 0) + V(1, 0, 0));
        const float us_ = 0.5f * (U(0, -1, 0) + U(0, 0, 0)) * 0.5f * (V(0, -1, 0) + V(1, -1, 0));
        const float ut = 0.5f * (U(0, 0, 0) + U(0, 0, 1)) * 0.5f * (W(0, 0, 0) + W(1, 0, 0));
        const float ub = 0.5f * (U(0, 0, -1) + U(0, 0, 0)) * 0.5f * (W(0, 0, -1) + W(1, 0, -1));
        float f = -r * ((ue * ue - uw * uw) + (un - us_) + (ut - ub));
        if (fl & FACE_U) {
            const float g = gu[c] + dt * U(0, 0, 0);
            gu[c] = g;
            f += q.alpha * g + q.beta * U(0, 0, 0);
        }
        f += r * ((T11(1, 0, 0) - T11(0, 0, 0)) + (t12 - T12(0, -1, 0)) + (t13 - T13(0, 0, -1)));
        const float fo = fuo_c;
        us[c] = U(0, 0, 0) + dt * (first ? f : 1.5f * f - 0.5f * fo);
        fuo[c] = f;
    }
    // ---- v face (i, j+1/2, k)
    {
        const float ve = 0.5f * (V(0, 0, 0) + V(1, 0, 0)) * 0.5f * (U(0, 0, 0) + U(0, 1, 0));
        const float vw = 0.5f * (V(-1, 0, 0) + V(0, 0, 0)) * 0.5f * (U(-1, 0, 0) + U(-1, 1, 0));
        const float vn = 0.5f * (V(0, 0, 0) + V(0, 1, 0)), vs_ = 0.5f * (V(0, -1, 0) + V(0, 0, 0));
        const float vt = 0.5f * (V(0, 0, 0) + V(0, 0, 1)) * 0.5f * (W(0, 0, 0) + W(0, 1, 0));
        const float vb = 0.5f * (V(0, 0, -1) + V(0, 0, 0)) * 0.5f * (W(0, 0, -1) + W(0, 1, -1));
        float f = -r * ((ve - vw) + (vn * vn - vs_ * vs_) + (vt - vb));
        if (fl & FACE_V) {
            const float g = gv[c] + dt * V(0, 0, 0);
            gv[c] = g;
            f += q.alpha * g + q.beta * V(0, 0, 0);
        }
        f += r * ((t12 - T12(-1, 0, 0)) + (T22(0, 1, 0) - T22(0, 0, 0)) + (t23 - T23(0, 0, -1)));
        const float fo = fvo_c;
        vs[c] = V(0, 0, 0) + dt * (first ? f : 1.5f * f - 0.5f * fo);
        fvo[c] = f;
    }
    // ---- w face (i, j, k+1/2)
    if (k < d.nz) {
        const float we = 0.5f * (W(0, 0, 0) + W(1, 0, 0)) * 0.5f * (U(0, 0, 0) + U(0, 0, 1));
        const float ww = 0.5f * (W(-1, 0, 0) + W(0, 0, 0)) * 0.5f * (U(-1, 0, 0) + U(-1, 0, 1));
        const float wn = 0.5f * (W(0, 0, 0) + W(0, 1, 0)) * 0.5f * (V(0, 0, 0) + V(0, 0, 1));
        const float ws_ = 0.5f * (W(0, -1, 0) + W(0, 0, 0)) * 0.5f * (V(0, -1, 0) + V(0, -1, 1));
        const float wt = 0.5f * (W(0, 0, 0) + W(0, 0, 1)), wb = 0.5f * (W(0, 0, -1) + W(0, 0, 0));
        float f = -r * ((we - ww) + (wn - ws_) + (wt * wt - wb * wb));
        if (fl & FACE_W) {
            const float g = gw[c] + dt * W(0, 0, 0);
            gw[c] = g;
            f += q.alpha * g + q.beta * W(0, 0, 0);
        }
        f += r * ((t13 - T13(-1, 0, 0)) + (t23 - T23(0, -1, 0)) + (T33(0, 0, 1) - T33(0, 0, 0)));
        const float fo = fwo_c;
        ws[c] = W(0, 0, 0) + dt * (first ? f : 1.5f * f - 0.5f * fo);
        fwo[c] = f;
    }
    if (i == 1) us[c - 1] = U(-1, 0, 0);  // the inflow face travels with u*
}

// The fused predictor: reads u^n (after velnw, interior faces only) and
// the inflow profile, writes u* to the other buffer set, nu_t of the
// interior, and updates F_old and the Goldstein integrals in place.
// Plane step k stores velocity plane k+2 (read from global memory during
// the previous step) into the slot of plane k-3 (its last reader, the
// predictor of plane k-2, finished before the previous step's barriers),
// issues the global reads of plane k+3 and of the step's own face flags and
// F_old, forms nu_t of plane k+1 in the slot of plane k-2 (last read by the
// predictor of plane k-1, before this step's first barrier) and predicts
// plane k: the global reads' latency hides behind the nu_t and predictor
// stages.
// grid (ceil(nx / LT_X), ceil(ny / LT_Y), ceil(nz / LT_KZ)), block LT_THREADS.
__global__ void __launch_bounds__(LT_THREADS)
les_predict_tile_kernel(LDev q, int first, const float *__restrict__ u, const float *__restrict__ v,
                        const float *__restrict__ w, const float *__restrict__ uin,
                        const uint8_t *__restrict__ face, float *__restrict__ nut, float *__restrict__ us,
                        float *__restrict__ vs, float *__restrict__ ws, float *__restrict__ fuo,
                        float *__restrict__ fvo, float *__restrict__ fwo, float *__restrict__ gu,
                        float *__restrict__ gv, float *__restrict__ gw)
{
    __shared__ LesTileSmem sm;
    const PDims &d = q.d;
    const int i0 = blockIdx.x * LT_X, j0 = blockIdx.y * LT_Y, k0 = blockIdx.z * LT_KZ;
    const int k1 = min(k0 + LT_KZ, d.nz);  // planes k0+1 .. k1 are predicted here
    const int tx = threadIdx.x % LT_X, ty = threadIdx.x / LT_X;
    const int i = i0 + 1 + tx, j = j0 + 1 + ty;
    const bool own = i <= d.nx && j <= d.ny;
    const int o = (ty + 2) * LT_HX + tx + 2;  // the cell in a velocity plane
    const int on = (ty + 1) * LT_EX + tx + 1;  // and in a nu_t plane
    const LtMap m = lt_map(d, i0, j0);
    // prologue: velocity planes k0-1 .. k0+2, nu_t planes k0 and k0+1
    for (int kk = k0 - 1; kk <= k0 + 2; ++kk) lt_store_plane(sm, lt_fetch_plane(q, m, kk, u, v, w, uin), kk);
    LtVel ahead = lt_fetch_plane(q, m, k0 + 3, u, v, w, uin);
    __syncthreads();
    lt_nut_plane(q, sm, m, k0, false, nut);
    lt_nut_plane(q, sm, m, k0 + 1, true, nut);
    for (int k = k0 + 1; k <= k1; ++k) {
        uint8_t fl = 0;
        float fuo_c = 0.0f, fvo_c = 0.0f, fwo_c = 0.0f;
        if (own && LES_OK(d, L(d, i, j, k)) && LES_OK(d, L(d, i, j, k) - 1)) {  // the predictor's own global reads, issued first
            const long long c = L(d, i, j, k);
            fl = face[c];
            fuo_c = fuo[c];
            fvo_c = fvo[c];
            fwo_c = fwo[c];
        }
        lt_store_plane(sm, ahead, k + 2);
        __syncthreads();
        if (k + 1 <= k1) ahead = lt_fetch_plane(q, m, k + 3, u, v, w, uin);  // consumed by the next plane step
        lt_nut_plane(q, sm, m, k + 1, k + 1 <= k1, nut);
        __syncthreads();
        if (own && LES_OK(d, L(d, i, j, k)) && LES_OK(d, L(d, i, j, k) - 1))
            lt_predict_cell(q, sm, k, i, j, o, on, first != 0, fl, fuo_c, fvo_c, fwo_c, us, vs, ws, fuo, fvo, fwo, gu,
                            gv, gw);
    }
}

// b = div(u*) / dt at interior cells.
__global__ void les_rhs_kernel(LDev q, const float *__restrict__ u, const float *__restrict__ v,
                               const float *__restrict__ w, float *__restrict__ b)
{
    const PDims &d = q.d;
    const int i = blockIdx.x * blockDim.x + threadIdx.x + 1;
    const int j = blockIdx.y + 1, k = blockIdx.z + 1;
    if (i > d.nx) return;
    const long long c = L(d, i, j, k), cs = L(d, i, (j > 1) ? j - 1 : d.ny, k);
    if (!LES_OK(d, c) || !LES_OK(d, c - 1) || !LES_OK(d, cs) || !LES_OK(d, c - d.plane)) return;
    const float vs = v[cs];
    const float wb = k > 1 ? w[c - d.plane] : 0.0f;  // the ground face is closed
    b[c] = q.rdxdt * ((u[c] - u[c - 1]) + (v[c] - vs) + (w[c] - wb));
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
    void *host_stage;      // pinned staging buffer of field copies to / from pageable memory
    size_t host_stage_bytes;
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
    const dim3 gt(ceil_div(d.nx, LT_X), ceil_div(d.ny, LT_Y), ceil_div(d.nz, LT_KZ));
    les_predict_tile_kernel<<<gt, LT_THREADS, 0, s->stream>>>(q, s->step == 0, u, v, w, s->uin, s->face, s->nut,
                                                              s->U[bset], s->V[bset], s->W[bset], s->fuo, s->fvo,
                                                              s->fwo, s->gu, s->gv, s->gw);
    les_rhs_kernel<<<g1, b1, 0, s->stream>>>(q, s->U[bset], s->V[bset], s->W[bset], s->b);
    GBSW_LAUNCH_CHECK();
    s->cur = bset;
    return GBSW_OK;
}

// True for host memory the copy engines reach directly (pinned or mapped).
bool host_is_pinned(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // plain pageable memory on some drivers: not an error of this context
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

gbsw_status ensure_host_stage(gbsw_les *s, size_t bytes)
{
    if (bytes <= s->host_stage_bytes) return GBSW_OK;
    if (s->host_stage) cudaFreeHost(s->host_stage);
    s->host_stage = nullptr;
    s->host_stage_bytes = 0;
    // the largest field (the FP64 pressure), so that one allocation serves every field
    const size_t want = std::max(bytes, (size_t)(s->q.d.nx + 2) * (s->q.d.ny + 2) * (s->q.d.nz + 2) * sizeof(double));
    if (cudaHostAlloc(&s->host_stage, want, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        s->host_stage = nullptr;
        return GBSW_ERR_OOM;
    }
    s->host_stage_bytes = want;
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
    s->solver.set_predicted_checks(true);
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
            s->solver.invalidate_stencil_cache();  // the guess changes p_hi before the solve
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
    const size_t elt = field == GBSW_LES_P ? sizeof(double) : sizeof(float);
    const void *src = field == GBSW_LES_P ? (const void *)s->solver.p_hi : (const void *)field_f32(s, field);
    if (!src) return GBSW_ERR_ARG;
    const size_t rows = (size_t)(d.ny + 2) * (size_t)(d.nz + 2), width = (size_t)(d.nx + 2) * elt;
    const bool direct = host_is_pinned(host);
    if (!direct) {
        const gbsw_status st = ensure_host_stage(s, width * rows);
        if (st != GBSW_OK) return st;
    }
    GBSW_CUDA_TRY(cudaMemcpy2DAsync(direct ? host : s->host_stage, width, src, d.pitch * elt, width, rows,
                                    cudaMemcpyDeviceToHost, s->stream));
    GBSW_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (!direct) memcpy(host, s->host_stage, width * rows);
    return GBSW_OK;
}

gbsw_status les_set_field(gbsw_les *s, int field, const void *host)
{
    if (!s || !host) return GBSW_ERR_ARG;
    const PDims &d = s->q.d;
    const size_t elt = field == GBSW_LES_P ? sizeof(double) : sizeof(float);
    void *dst = field == GBSW_LES_P ? (void *)s->solver.p_hi : (void *)field_f32(s, field);
    if (!dst) return GBSW_ERR_ARG;
    if (field == GBSW_LES_P) s->solver.invalidate_stencil_cache();
    const size_t rows = (size_t)(d.ny + 2) * (size_t)(d.nz + 2), width = (size_t)(d.nx + 2) * elt;
    const bool direct = host_is_pinned(host);
    if (!direct) {
        const gbsw_status st = ensure_host_stage(s, width * rows);
        if (st != GBSW_OK) return st;
        memcpy(s->host_stage, host, width * rows);
    }
    GBSW_CUDA_TRY(cudaMemcpy2DAsync(dst, d.pitch * elt, direct ? host : s->host_stage, width, width, rows,
                                    cudaMemcpyHostToDevice, s->stream));
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

gbsw_status les_set_check_prediction(gbsw_les *s, int on)
{
    if (!s) return GBSW_ERR_ARG;
    s->solver.set_predicted_checks(on != 0);
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
    if (s->host_stage) cudaFreeHost(s->host_stage);
    s->solver.release();
    delete s;
}

}  // extern "C"

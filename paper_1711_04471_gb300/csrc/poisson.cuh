// Pressure Poisson solver of the UFLES step ("press", Sec. 6.3.1 of
// arXiv:1711.04471: the Poisson equation for pressure solved by successive
// over-relaxation), red-black ordered, FP32 sweeps with an FP64 outer
// residual.
//
// Operator (7-point Laplacian on an nx*ny*nz cell grid of spacing dx):
//   (A p)_c = (sum of neighbour values - d_c p_c) / dx^2,
//   d_c = 6 - [i == 1] - [k == 1] - [k == nz] + [i == nx]
// i.e. Neumann at the inflow plane, the ground and the lid (mirror ghost),
// Dirichlet p = 0 on the outflow face (antisymmetric ghost), periodic in y.
//
// Mixed precision without changing the iteration: SOR is an affine
// stationary method, so running it on the correction e for A e = r with
// r = b - A p_hi from e = 0 produces p_hi + e equal (in exact arithmetic) to
// the SOR iterates on p itself.  Every m iterations the FP64 residual
// r = b - A (p_hi + e) and its norm are formed, and e is folded into the
// FP64 base p_hi by the next sweep.  The sweeps move 4-byte words only; the
// 1e-6 relative residual is reachable although FP32 storage of p alone
// would floor it near 1e-5 for smooth pressure fields.
//
// Device layout.  p_hi: (nz+2) x (ny+2) x pitch FP64, interior cell
// (i,j,k) (1-based) at k*plane + j*pitch + i.  e and r are stored split by
// colour c = (i+j+k) mod 2: colour array c holds cell (i,j,k) of that
// colour at k*cplane + j*cpitch + SOR_SLOT0 + ((i-1) >> 1), so a half-sweep
// reads its own colour and the other colour with unit stride, and slot 0
// of every row starts a 16-byte word group.  The SOR_SLOT0 words before
// slot 0, the slots past the last cell of a row (at least four), and the
// y/z ghost rows stay 0: the boundary rules enter only through d_c, and y
// is wrapped explicitly.
#pragma once

#include "common.cuh"

namespace gbsw {

struct PDims {
    int nx, ny, nz, pitch;
    long long plane;   // (ny+2) * pitch
    int cpitch;        // row pitch of a colour array: SOR_SLOT0 + round_up((nx+1)/2, 4) + 4
    long long cplane;  // (ny+2) * cpitch
    double dx;
    double rdx2;       // 1 / dx^2, formed once on the host (an FP64 division per thread costs dozens of FP64 operations)
};

struct PoissonCtl {
    double bb;        // ||b||^2
    double rr;        // ||r||^2 at the last check
    double rho;       // ||r|| / ||b||
    int iters;        // SOR iterations done
    int done;
    int status;       // DEV_* code
    int next;         // predicted checks: iterations from the last check to the next
    double rho_prev;  // predicted checks: rho and iters at the check before the last
    int iters_prev;
    int since;        // predicted checks: iterations since the last check
};

class PoissonSolver {
public:
    // b: device array in the padded layout (owned by the caller), read at
    // every residual check.  p_hi is owned by the solver.
    gbsw_status init(int nx, int ny, int nz, double dx, const float *b, cudaStream_t stream);
    void release();
    gbsw_status configure(double omega, double tol, int max_iter, int check_every);
    // Predicted checks: after a check, the next one comes at the iteration
    // where the convergence rate measured between the last two checks
    // reaches the tolerance (with a small margin), rounded up to a whole
    // chunk of the loop body (the largest divisor of check_every up to
    // SOR_CHUNK_MAX), and never later than check_every iterations.  The
    // iterates and the stopping test are unchanged; only where the test is
    // taken moves.  Off: a test every check_every iterations.
    void set_predicted_checks(bool on);
    // Enqueue one solve (asynchronous; one graph launch).
    gbsw_status enqueue();
    // Enqueue exactly niter iterations with no convergence test (the
    // paper's fixed-count SOR); the control block receives the final
    // residual.  With use_graph (a solver that is used again) and niter up
    // to SOR_FIXED_GRAPH_MAX_ITER, the sequence is captured once into a
    // CUDA graph and replayed; otherwise its kernels are launched directly.
    gbsw_status enqueue_fixed(int niter, bool use_graph);
    // Copy the control block of the last solve into *out (device -> device).
    gbsw_status record(PoissonCtl *dev_dst);
    // p_hi was changed outside a solve: the next fixed-count solve forms its
    // first residual's stencil afresh instead of reusing the stored one.
    void invalidate_stencil_cache() { s_valid_ = false; }

    PDims d{};
    double *p_hi = nullptr;   // FP64 pressure (the solution)
    float *e[2] = {};         // FP32 correction of the inner sweeps, per colour
    float *r[2] = {};         // FP32 residual (right-hand side of the sweeps), per colour
    const float *b = nullptr;
    double *partials = nullptr;   // 2 per residual block (||r||^2, ||b||^2)
    dim3 rgrid;                   // residual grid: (ceil(nx/256), ny, ceil(nz/8)), fixed per size
    int rblocks = 0;
    PoissonCtl *ctl = nullptr;
    double *s_cache = nullptr;    // fixed-count solves: stencil of p_hi stored by the final residual
    int *s_ok = nullptr;          // device flag: s_cache matches p_hi
    cudaStream_t stream = nullptr;
    double omega = 1.8, tol = 1e-6;
    int max_iter = 100000, m = 10;

private:
    gbsw_status build_graph();
    gbsw_status build_graph_predicted();
    gbsw_status record_fixed(int niter, cudaStream_t s);
    cudaGraphExec_t fixed_exec_ = nullptr;
    int fixed_niter_ = -1;
    bool fixed_dirty_ = true;
    cudaGraph_t graph_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
    bool dirty_ = true;
    bool predict_ = false;
    bool s_valid_ = false;  // host view of s_ok for the next fixed-count solve
};

constexpr int POI_RES_PLANES = 16;    // z-planes per thread of the residual kernel
constexpr int SOR_SLOT0 = 4;          // offset of slot 0 in a colour row (keeps float4 groups aligned)
constexpr int SOR_THREADS = 128;      // threads per block of the SOR sweep
constexpr int SOR_KZ = 2;             // z-planes per thread of the SOR sweep
constexpr int SOR_FIXED_GRAPH_MAX_ITER = 1000;   // longest fixed-count solve captured into a graph
constexpr int SOR_CHUNK_MAX = 50;     // predicted checks: iterations per loop body at most
constexpr int POI_RED_THREADS = 256;

// The values 4, 5, 6, 7 that the diagonal d_c takes, and their reciprocals
// rounded to FP32 (y = RN(1/d), formed by an IEEE division on the host).
struct SorDiag {
    float d[4];
    float y[4];
};

inline SorDiag sor_diag()
{
    SorDiag g;
    for (int n = 0; n < 4; ++n) {
        g.d[n] = (float)(4 + n);
        g.y[n] = 1.0f / g.d[n];
    }
    return g;
}

// x / d rounded to nearest even, for d in {4, 5, 6, 7} and y = RN(1/d):
// q = RN(x y) is within one unit in the last place of x / d, the remainder
// x - q d is then exact in one FMA, and q + (x - q d) y rounded once is the
// correctly rounded quotient (the correction step of P. Markstein, "IA-64
// and Elementary Functions", Prentice Hall 2000, ch. 8).  When the
// remainder is zero, q is the quotient as it stands (this keeps the sign
// of a zero x).  A non-finite x gives a NaN (the residual check reports
// it).  gbsw_selftest_sor_division compares it with the IEEE division for
// every finite FP32 x.
__device__ __forceinline__ float sor_div(float x, float d, float y)
{
    const float q = __fmul_rn(x, y);
    const float r = __fmaf_rn(-q, d, x);
    return r == 0.0f ? q : __fmaf_rn(r, y, q);
}

}  // namespace gbsw

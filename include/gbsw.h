/*
 * gbsw.h -- C ABI of the GB300 (sm_103a) time-step library for the two
 * programs evaluated in Vanderbauwhede & Davidson, "Domain-Specific
 * Acceleration and Auto-Parallelization of Legacy Scientific Code in
 * FORTRAN 77 using Source-to-Source Compilation" (arXiv:1711.04471):
 * the 2-D shallow-water model (Sec. 6.2) and the Large Eddy Simulator for
 * Urban Flows (Sec. 6.3).
 *
 * General rules
 *  - Every call returns a gbsw_status; 0 is success, negative is an error,
 *    positive is a non-fatal condition.  Nothing is asserted or trapped on
 *    the device: kernels record problems in a device status word that the
 *    next synchronising call reports.
 *  - Host arrays are row-major with x fastest.  Host inputs to *_create are
 *    FP64 and are converted to the FP32 device state once; afterwards the
 *    state stays resident in device memory across steps (Sec. 4.3: data
 *    are moved to the device once, not per kernel call).
 *  - A context owns all device memory it allocates.  Entry points that take
 *    device pointers say so; the caller owns those buffers.
 *  - `stream` is a cudaStream_t passed as void*; NULL selects the legacy
 *    default stream.  Calls on one context are not thread-safe.  The library
 *    also fills a few process-wide caches on first use (the SM count of the
 *    device current at the first call, each kernel's resident blocks per SM,
 *    the convolutions' shared-memory attributes): make the first call of
 *    each kind from one host thread, on devices of one model.
 *  - Asynchronous calls (sw_step, ...) enqueue work and return; errors of
 *    the enqueued kernels surface at the next synchronising call.
 */
#ifndef GBSW_H
#define GBSW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GBSW_OK = 0,
    GBSW_ERR_ARG = -1,          /* invalid argument or size */
    GBSW_ERR_CUDA = -2,         /* a CUDA runtime call failed */
    GBSW_ERR_OOM = -3,          /* device or pinned allocation failed */
    GBSW_ERR_CFL = -4,          /* time step violates the gravity-wave CFL limit */
    GBSW_ERR_NONFINITE = -5,    /* a reduction met NaN or Inf in the state */
    GBSW_ERR_TIMEOUT = -6,      /* a bounded device-side wait gave up */
    GBSW_ERR_DEVICE_BOUNDS = -7,/* a kernel detected an out-of-range index */
    GBSW_NOT_CONVERGED = 1      /* iterative solve stopped at max_iter */
} gbsw_status;

/* Human-readable name of a status code (static string). */
const char *gbsw_status_string(int status);

/* Library version, as major*10000 + minor*100 + patch. */
int gbsw_version(void);

/* Text of the last CUDA failure seen by this thread (static buffer, empty
 * if none). */
const char *gbsw_last_error(void);

/*
 * Measurement: copy bandwidth of data that stays in L2.  Copies one device
 * buffer of `bytes` bytes (>= 1 MiB, a multiple of 16) onto another,
 * `passes` times inside one launch of one wave of blocks, and writes the
 * best of five timed launches (after one that brings both buffers into L2)
 * to *gbs in GB/s, counting read and write bytes.  With 2 x bytes well
 * below the L2 size this is the ceiling of a kernel whose working set stays
 * in L2 (the SOR sweeps of the pressure solve, Sec. 6.3.1 "press").
 * Allocates and frees its buffers; synchronous on the default stream.
 */
gbsw_status gbsw_measure_l2_copy(long long bytes, int passes, double *gbs);

/*
 * Bounds-checked debug build (a stand-in for a memory-checking sanitizer;
 * the paper has no counterpart).  libgbsw_debug.so, built from the same
 * sources with GBSW_DEBUG_BOUNDS=1, tests the global indices of the 2DSW
 * kernels (the streaming, tile and ensemble kernels), of the SOR sweep, of
 * the UFLES velnw, predictor and right-hand-side kernels and of the warm
 * start's grid transfers against their buffers' extents before the
 * access; a failed test skips the access and is counted, so a wrong index
 * never faults.  gbsw_debug_bounds writes the
 * count since the last call to *violations (and clears it), returning
 * GBSW_ERR_DEVICE_BOUNDS if it is not 0; in the product build it writes -1
 * and returns GBSW_OK.  Synchronises the device.
 */
gbsw_status gbsw_debug_bounds(long long *violations);

/* Self-test of that index test: checks index n of an n-element device
 * buffer (no access is made) and returns GBSW_ERR_DEVICE_BOUNDS when the
 * violation was counted, in either build.  Synchronous. */
gbsw_status gbsw_selftest_bounds(void);

/* Self-test of the bounded device-side waits (the paper has no
 * counterpart).  which = 0 waits on an mbarrier phase that never completes
 * for `budget` clock cycles, which = 1 spins on a flag that is never set
 * for `budget` iterations; 1 <= budget <= 1e9.  Returns GBSW_ERR_TIMEOUT
 * when the wait gave up as designed, leaving the context usable.
 * Synchronous. */
gbsw_status gbsw_selftest_wait(int which, long long budget);

/* Self-test of the division by the Poisson operator's diagonal inside the
 * SOR sweep (the paper has no counterpart): the sweep divides by
 * d in {4, 5, 6, 7} through a rounded reciprocal and one FMA correction;
 * this runs it on the device for every finite FP32 x and compares it bit
 * for bit with the IEEE division x / d.  counts (host, 3 entries) receives
 * the mismatches with |x| >= 2^-100, the mismatches with smaller |x|, and
 * the smallest mismatching bit pattern (0xffffffff if none).  d outside
 * 4..7 or a NULL counts gives GBSW_ERR_ARG.  Synchronous; about 4e9
 * divisions. */
gbsw_status gbsw_selftest_sor_division(int d, unsigned long long *counts);

/* ------------------------------------------------------------------------
 * 2-D shallow water (Sec. 6.2: time loop of predictor "dyn", first-order
 * Shapiro filter "shapiro", then the velocity/state update).
 *
 * Grid: staggered C-grid of nx*ny interior cells with closed walls.
 * Surface elevation eta and still-water depth H at cell centres, u on the
 * east face and v on the north face of each cell.  Per step:
 *   u' = u - g dt d(eta)/dx (likewise v'), kept only where the face is
 *        wet on both sides or flow leaves a wet cell, else 0;
 *   eta* = eta - dt div(upwind flux u' h), h = H + eta;
 *   eta+ = masked 5-point Shapiro filter of eta* with weight eps on wet
 *          cells; wet = (H + eta > hmin).
 * ---------------------------------------------------------------------- */

typedef struct gbsw_sw gbsw_sw;

typedef struct {
    int nx, ny;          /* interior cells, each >= 2 */
    double dx, dy;       /* cell size (m), > 0 */
    double dt;           /* time step (s), > 0 */
    double g;            /* gravity (m/s^2), e.g. 9.81 */
    double eps;          /* Shapiro filter weight, 0 <= eps <= 1 (e.g. 0.05) */
    double hmin;         /* wet threshold (m): wet iff H + eta > hmin */
} gbsw_sw_params;

/*
 * Create a 2DSW context and upload the initial state.
 *   H     host, ny*nx FP64 still-water depth (m), negative = land
 *   eta0  host, ny*nx FP64 initial elevation (m); values below -H are
 *         raised to -H; u = v = 0 initially.
 * Fails with GBSW_ERR_CFL if sqrt(g*max(H+eta0)) * dt * sqrt(1/dx^2+1/dy^2)
 * exceeds 1, GBSW_ERR_ARG on bad sizes or NULL pointers.  *out is set only
 * on success.  Synchronous.
 */
gbsw_status sw_create(const gbsw_sw_params *params, const double *H, const double *eta0,
                      void *stream, gbsw_sw **out);

/* Advance the state by nsteps >= 0 time steps.  Asynchronous on the
 * context stream; several steps are fused per kernel launch. */
gbsw_status sw_step(gbsw_sw *sw, int nsteps);

/*
 * Total volume dx*dy*sum(H + eta) over interior cells, and the part held
 * by wet cells, accumulated in FP64 on the device in a fixed order (the
 * result is bitwise reproducible).  Either output may be NULL.  Host
 * outputs; synchronises the context stream.  Returns GBSW_ERR_NONFINITE
 * if any interior eta is NaN or Inf.
 */
gbsw_status sw_volume(gbsw_sw *sw, double *volume, double *wet_volume);

/*
 * Copy the state to host buffers (any may be NULL): eta ny*nx, u ny*(nx+1)
 * (east faces i = 0..nx, the two wall columns are 0), v (ny+1)*nx (north
 * faces j = 0..ny, wall rows 0), wet ny*nx bytes (1 = wet).  Synchronous.
 */
gbsw_status sw_get_state(gbsw_sw *sw, float *eta, float *u, float *v, uint8_t *wet);

/* Replace the state from host buffers in the layout of sw_get_state (wall
 * faces are ignored and kept 0).  Any of eta, u, v may be NULL to keep the
 * current field.  Synchronous. */
gbsw_status sw_set_state(gbsw_sw *sw, const float *eta, const float *u, const float *v);

/* Number of time steps fused per kernel launch (temporal blocking depth):
 * 0 = automatic, else 1..6 (the row-segment height returns to automatic). */
gbsw_status sw_set_blocking(gbsw_sw *sw, int steps_per_launch);

/* Tiling of the fused kernel: steps per launch (0 = automatic, else 1..6)
 * and the row-segment height of a thread block of the streaming kernel (0 =
 * automatic: one wave of resident blocks, segments of at least 8T rows),
 * or rows < 0 for the tile kernel, made for grids that fit in L2: a block
 * holds 32 columns x h rows and a 2T-cell halo in shared memory, with
 * h = 32 for rows = -1 and h = -rows for rows <= -2 (T = 1..3 given
 * explicitly; h at most 52, 43, 34 for T = 1, 2, 3, else GBSW_ERR_ARG).
 * Results do not depend on the tiling (every operation is rounded as
 * written). */
gbsw_status sw_set_tiling(gbsw_sw *sw, int steps_per_launch, int rows);

/* Choose the tiling by measurement: times trial_steps (1..100000, rounded
 * to whole launches) on the context's own state for each depth T = 1..6
 * and row-segment heights giving the default, one, two and three waves of
 * resident blocks, and the tile kernel for T = 1..3 with 32-row tiles and
 * with the tile height that spreads its blocks most evenly over the SMs,
 * keeps the fastest (written to *T_out, *rows_out in the encoding of
 * sw_set_tiling, if non-NULL) and restores the state exactly.  Allocates a copy of the state;
 * synchronous.  The paper's grids (Sec. 6.2: 500^2 to 2000^2) are small
 * enough to stay in L2, where the best tiling differs from the 4096^2
 * default. */
gbsw_status sw_autotune(gbsw_sw *sw, int trial_steps, int *T_out, int *rows_out);

/* Release the context and its device memory.  NULL is ignored. */
void sw_destroy(gbsw_sw *sw);

/* ------------------------------------------------------------------------
 * 2DSW in FP64 end to end (Sec. 6.2: the time loop of "dyn" and "shapiro",
 * which the paper's compiler turns into three map kernels; the paper does
 * not state the precision).  The same method, parameters and conventions
 * as sw_* above, run as three kernels per step (momentum on the faces,
 * continuity on the cells, masked Shapiro filter) with every FP64
 * operation in the order written in the formulas above and rounded as
 * written (no multiply-add contraction), so the state is a deterministic
 * function of the inputs.  Slower than sw_step (FP64 throughput and no
 * temporal blocking); meant for precision studies.
 * ---------------------------------------------------------------------- */

typedef struct gbsw_sw64 gbsw_sw64;

/* As sw_create (same arguments, checks and errors), keeping H, eta, u, v
 * in FP64 on the device. */
gbsw_status sw64_create(const gbsw_sw_params *params, const double *H, const double *eta0,
                        void *stream, gbsw_sw64 **out);

/* Advance by nsteps >= 0 time steps (3 kernel launches per step,
 * asynchronous on the context stream). */
gbsw_status sw64_step(gbsw_sw64 *sw, int nsteps);

/* As sw_volume: dx*dy*sum(H + eta) and the wet part, FP64 on the device in
 * a fixed order; GBSW_ERR_NONFINITE if any eta is NaN or Inf.  Syncs. */
gbsw_status sw64_volume(gbsw_sw64 *sw, double *volume, double *wet_volume);

/* As sw_get_state with FP64 host buffers (any may be NULL): eta ny*nx,
 * u ny*(nx+1), v (ny+1)*nx, wet ny*nx bytes.  Synchronous. */
gbsw_status sw64_get_state(gbsw_sw64 *sw, double *eta, double *u, double *v, uint8_t *wet);

/* Release the context.  NULL is ignored. */
void sw64_destroy(gbsw_sw64 *sw);

/* ------------------------------------------------------------------------
 * Batched 2DSW ensemble: n independent instances (each its own size,
 * bathymetry and initial state) of the 2DSW step above, advanced together.
 * The paper has no ensemble; this is the step of Sec. 6.2 applied to many
 * grids at once.  One sw_batch_step call is one CUDA-graph launch of a
 * persistent cooperative kernel that processes every instance's tiles
 * level after level (a level = steps_per_level fused time steps), with a
 * bounded grid barrier between levels.
 * ---------------------------------------------------------------------- */

typedef struct gbsw_sw_batch gbsw_sw_batch;

/* params, H[m], eta0[m]: n entries, each as in sw_create (host, FP64,
 * ny*nx).  Synchronous. */
gbsw_status sw_batch_create(int n, const gbsw_sw_params *params, const double *const *H,
                            const double *const *eta0, void *stream, gbsw_sw_batch **out);

/* Advance every instance by nsteps (asynchronous; one graph launch, cached
 * per nsteps). */
gbsw_status sw_batch_step(gbsw_sw_batch *b, int nsteps);

/* The same steps issued as one launch per instance and fused level (the
 * unbatched baseline the persistent kernel is measured against). */
gbsw_status sw_batch_step_separate(gbsw_sw_batch *b, int nsteps);

/* FP64 volumes (and wet volumes) of every instance into host arrays of n
 * (either may be NULL); synchronises; reports GBSW_ERR_TIMEOUT if a grid
 * barrier wait gave up, GBSW_ERR_NONFINITE on NaN/Inf. */
gbsw_status sw_batch_volumes(gbsw_sw_batch *b, double *volumes, double *wet_volumes);

/* Copy instance m's state to host buffers in the layout of sw_get_state. */
gbsw_status sw_batch_get_state(gbsw_sw_batch *b, int m, float *eta, float *u, float *v);

/* Tiling: fused steps per level (1..4) and rows per work item (8..65536). */
gbsw_status sw_batch_set_tiling(gbsw_sw_batch *b, int steps_per_level, int rows_per_item);
gbsw_status sw_batch_get_tiling(gbsw_sw_batch *b, int *steps_per_level, int *rows_per_item);

/* Time every (steps_per_level, rows_per_item) candidate on this batch
 * (state saved and restored), keep the fastest and return it.  If
 * cache_path is not NULL the choice is looked up in / appended to that
 * text file, keyed by device name and instance sizes. */
gbsw_status sw_batch_autotune(gbsw_sw_batch *b, int trial_steps, const char *cache_path, int *steps_per_level,
                              int *rows_per_item);

void sw_batch_destroy(gbsw_sw_batch *b);

/* ------------------------------------------------------------------------
 * Urban LES (Sec. 6.3.1: each step runs velnw, bondv1, velfg, feedbf, les,
 * adam and press, in that order).
 *
 * Grid: nx*ny*nz cubic cells of size dx; u on east faces (x = 0 inflow
 * plane, x = nx*dx outflow plane), v on north faces (periodic in y), w on
 * top faces (ground and lid closed); pressure at centres.  Per step:
 *   velnw : u = u* - dt grad p (previous pressure; p = 0 on the outflow face)
 *   bondv1: inflow u = u_ref ln(z/z0)/ln(z_ref/z0), v = w = 0 at the inflow,
 *           zero gradient at the outflow, periodic in y, no slip at the
 *           ground, free slip at the lid
 *   velfg : F = -div(u u) (flux form, second-order central)
 *   feedbf: faces touching a building cell: G += dt u, F += alpha G + beta u
 *           (Goldstein feedback forcing)
 *   les   : nu_t = (cs dx)^2 sqrt(2 S:S); F += div(2 (nu + nu_t) S)
 *   adam  : u* = u + dt (3/2 F - 1/2 F_old) (forward Euler on step 0)
 *   press : A p = div(u*)/dt by red-black SOR (relaxation omega) from the
 *           previous pressure, until ||b - A p||_2 <= tol ||b||_2 (FP64
 *           norm, tested on the device every check_every iterations) or
 *           max_iter iterations.  A: 7-point Laplacian, Neumann at the
 *           inflow, ground and lid, Dirichlet p = 0 at the outflow face,
 *           periodic in y.
 * Velocities and the SOR sweeps are FP32; the pressure itself is kept in
 * FP64 (the sweeps iterate on an FP32 correction that is folded into it at
 * every residual check, which leaves the SOR iterates unchanged in exact
 * arithmetic).
 * ---------------------------------------------------------------------- */

typedef struct gbsw_les gbsw_les;

typedef struct {
    int nx, ny, nz;         /* cells; ny even (red-black colouring is periodic in y); each >= 2 */
    double dx;              /* cell size (m) */
    double dt;              /* time step (s) */
    double u_ref, z_ref;    /* inflow speed u_ref (m/s) at height z_ref (m) */
    double z0;              /* roughness length (m), 0 < z0 < dx/2 */
    double cs;              /* Smagorinsky constant (e.g. 0.1) */
    double nu;              /* molecular viscosity (m^2/s) */
    double alpha, beta;     /* Goldstein gains (s^-2, s^-1), both <= 0 */
    double omega;           /* SOR relaxation, 0 < omega < 2 */
    double tol;             /* relative residual target */
    int max_iter;           /* SOR iteration cap per step */
    int check_every;        /* iterations between FP64 residual checks, 1..1000 */
} gbsw_les_params;

typedef struct {
    int iters;              /* SOR iterations (a multiple of check_every) */
    int status;             /* GBSW_OK, GBSW_NOT_CONVERGED or an error */
    double rel_res;         /* final ||b - A p|| / ||b|| */
    float ms_predictor;     /* device time of velnw .. rhs */
    float ms_solve;         /* device time of the pressure solve */
    float ms_guess;         /* device time of the learned warm start (0 without) */
} gbsw_les_stats;

/* Field ids for les_get_field / les_set_field.  Every field is exchanged
 * in the padded layout (nz+2) x (ny+2) x (nx+2), x fastest, ghost layer
 * included; GBSW_LES_P is FP64, all others FP32.  U, V, W are the
 * predicted velocity u* that the next step projects. */
enum {
    GBSW_LES_U = 0, GBSW_LES_V = 1, GBSW_LES_W = 2, GBSW_LES_P = 3,
    GBSW_LES_FU_OLD = 4, GBSW_LES_FV_OLD = 5, GBSW_LES_FW_OLD = 6,
    GBSW_LES_GU = 7, GBSW_LES_GV = 8, GBSW_LES_GW = 9,
    GBSW_LES_NUT = 10, GBSW_LES_B = 11
};

/*
 * Create an LES context.  solid: host nz*ny*nx bytes (1 = building cell),
 * or NULL for none.  Initial state: u* = inflow profile on every x-face
 * that touches no building (0 on those that do), v* = w* = 0, p = 0.
 * GBSW_ERR_CFL if u_max dt/dx > 0.5 for the inflow profile.  Synchronous.
 */
gbsw_status les_create(const gbsw_les_params *params, const uint8_t *solid, void *stream, gbsw_les **out);

/*
 * Advance nsteps steps.  stats: host array of nsteps records or NULL.
 * Synchronises at the end; returns the worst per-step status
 * (GBSW_NOT_CONVERGED if any solve stopped at max_iter).
 */
gbsw_status les_step(gbsw_les *les, int nsteps, gbsw_les_stats *stats);

/* Copy one field to / from a host buffer (layout above).  Synchronous.
 * A pinned host buffer is read or written by the copy engine directly; a
 * pageable one goes through a pinned staging buffer of the context
 * (allocated on first use with the size of one padded field, freed by
 * les_destroy), because a pitched copy to pageable memory is two orders of
 * magnitude slower (61 ms against 0.4 ms for the 256x256x128 FP64
 * pressure on a GB300).  GBSW_ERR_OOM if the staging buffer cannot be
 * allocated. */
gbsw_status les_get_field(gbsw_les *les, int field, void *host);
gbsw_status les_set_field(gbsw_les *les, int field, const void *host);

/* Steps taken so far (step 0 uses forward Euler); settable for restarts. */
gbsw_status les_get_step(gbsw_les *les, int *step);
gbsw_status les_set_step(gbsw_les *les, int step);

/* The whole state that the next step depends on (Sec. 6.3.1: the
 * predicted velocity that velnw projects, the pressure, the previous
 * tendencies of adam and the time integrals of feedbf), as host buffers in
 * the padded layout above, plus the step count.  A NULL buffer is skipped. */
typedef struct {
    float *u, *v, *w;        /* u*, v*, w* */
    double *p;               /* pressure (FP64) */
    float *fu_old, *fv_old, *fw_old;
    float *gu, *gv, *gw;
    int step;
} gbsw_les_state;

/* Checkpoint and restart: copy the state out of / into the context.  The
 * next step from a restored state is bitwise the step the context would
 * have taken.  Synchronous. */
gbsw_status les_get_state(gbsw_les *les, gbsw_les_state *state);
gbsw_status les_set_state(gbsw_les *les, const gbsw_les_state *state);

/* Change the SOR parameters of later steps. */
gbsw_status les_set_solver(gbsw_les *les, double omega, double tol, int max_iter, int check_every);

/* Predicted convergence checks (on by default; on != 0).  SOR's residual
 * falls geometrically, so after each check the next one is placed at the
 * iteration where the rate measured between the last two checks reaches
 * the tolerance (with a 3 % + 1 iteration margin), never more than
 * check_every iterations on.  The solve loop runs chunks of iterations (the
 * largest divisor of check_every up to 50, or 50 when that divisor is
 * below 12) and takes the check at the first chunk boundary at or past
 * that point.  The iterates and the FP64 stopping test (Sec. 6.3.1, press)
 * are unchanged: a step stops at the first check whose residual is within
 * tol, as before, only with fewer wasted iterations between the tolerance
 * and the check.  Off: a check every check_every iterations.  The
 * standalone poisson_solve always checks every check_every iterations. */
gbsw_status les_set_check_prediction(gbsw_les *les, int on);

/* Paper mode (Sec. 6.3.2 runs UFLES with the number of SOR iterations set
 * to 50): niter > 0 makes every later step run exactly niter SOR
 * iterations with no convergence test (stats report the final residual,
 * status GBSW_OK); 0 restores the tolerance-driven solve. */
gbsw_status les_set_fixed_iterations(gbsw_les *les, int niter);

void les_destroy(gbsw_les *les);

/*
 * Stand-alone pressure solve with the operator of les_step.
 *   p  device, nz*ny*nx FP32 (x fastest): initial guess in, solution out
 *   b  device, nz*ny*nx FP32 right-hand side
 * Both are caller-owned.  ny must be even.  Iterations are counted in
 * multiples of check_every.  tol < 0 selects the fixed-count mode of the
 * paper: exactly max_iter iterations, no convergence test, GBSW_OK.  Synchronous on `stream`; returns GBSW_OK when
 * ||b - A p|| <= tol ||b|| (or ||b|| < 1e-30, with 0 iterations),
 * GBSW_NOT_CONVERGED at max_iter.  *iters and *rel_res may be NULL.
 * Allocates and frees its own workspace (FP64 pressure, FP32 correction
 * and residual).
 */
gbsw_status poisson_solve(int nx, int ny, int nz, double dx, float *p, const float *b, double omega, double tol,
                          int max_iter, int check_every, void *stream, int *iters, double *rel_res);

/* ------------------------------------------------------------------------
 * Learned warm start for the pressure solve: a 3-D convolutional U-Net
 * (not in the paper; SOR from Sec. 6.3.1 still decides the answer).  The
 * 3x3x3 convolutions run on the tensor cores (tcgen05, BF16 operands, FP32
 * accumulation in tensor memory).
 * ---------------------------------------------------------------------- */

/*
 * Operator-level entry points: each runs one of the network's kernels on
 * dense FP32 device tensors (nsamples, D, H, W, C), channels last, so that
 * it can be compared with an FP64 reference on its own.  Inputs are
 * rounded to BF16 (nearest even) as the network stores its activations;
 * results are the kernels' FP32 values.  Geometry rule of the tcgen05
 * convolutions: W a power of two or a multiple of 128; with m =
 * 128/min(W, 128), H a multiple of m, or H a power of two below m with
 * W*H >= 16 (a tile then spans m/H planes).  Each call allocates and frees
 * temporary device buffers and is synchronous on `stream`; bad sizes or
 * NULL pointers return GBSW_ERR_ARG.
 */

/*
 * One 3x3x3 convolution with zero padding:
 *   x     nsamples*D*H*W*cin, w 27*cout*cin with w[tap][co][ci], tap =
 *         (dz+1)*9 + (dy+1)*3 + (dx+1) for input offsets dz, dy, dx (both
 *         rounded to BF16), bias cout FP32 (epilogue 0 only)
 *   epilogue 0: y = max(conv + bias, 0); 1: y = conv; 2: y = conv where
 *         mask > 0, else 0 (mask: FP32, same shape as y)
 *   y     nsamples*D*H*W*cout FP32 (the FP32 accumulator)
 * (cin, cout) one of the network's pairs, (16|32|64, 16|32|64) but not
 * (64, 64), or cin = 2, which runs zero-padded to 16 as the first layer
 * does.
 */
gbsw_status unet_conv3d(int nsamples, int D, int H, int W, int cin, int cout, const float *x, const float *w,
                        const float *bias, int epilogue, const float *mask, float *y, void *stream);

/*
 * Backward-data of that convolution (the tcgen05 kernel with the flipped,
 * transposed weight pack): gx[v][ci] = sum over taps and co of
 * gy[v - off(tap)][co] w[tap][co][ci], zero outside the sample; with mask
 * non-NULL (FP32, shape of gx) gx = 0 where mask <= 0.  gy
 * nsamples*D*H*W*cout, w 27*cout*cin, gx nsamples*D*H*W*cin.  (cout, cin)
 * must be a pair unet_conv3d accepts with cin >= 16.
 */
gbsw_status unet_conv3d_bwd_data(int nsamples, int D, int H, int W, int cin, int cout, const float *gy,
                                 const float *w, const float *mask, float *gx, void *stream);

/*
 * Weight and bias gradients of that convolution on the tensor cores:
 * dw[tap][co][ci] = sum_v gy[v][co] x[v + off(tap)][ci] (zero outside the
 * sample), db[co] = sum_v gy[v][co]; dw (27*cout*cin) and db (cout) are
 * overwritten.  x nsamples*D*H*W*cin, gy nsamples*D*H*W*cout.  (cin, cout)
 * one of (2|16, 16), (16, 32), (32, 16|32|64), (64, 16|32): the network's
 * layers.
 */
gbsw_status unet_conv3d_bwd_weight(int nsamples, int D, int H, int W, int cin, int cout, const float *x,
                                   const float *gy, float *dw, float *db, void *stream);

/*
 * The glue between the convolutions, C in {8, 16, ..., 64}:
 *   op 0  out (n, D/2, H/2, W/2, C) = 2x2x2 average of a (n, D, H, W, C)
 *   op 1  out (n, 2D, 2H, 2W, C) = nearest upsampling of a (n, D, H, W, C)
 *   op 2  out (n, D, H, W, C) = sum of the 8 children in a (n, 2D, 2H, 2W, C)
 *         (the adjoint of op 1)
 *   op 3  out (n, D, H, W, C) = (a + b / 8 at the parent cell) * [c > 0],
 *         a, c (n, D, H, W, C), b (n, D/2, H/2, W/2, C): the gradient of a
 *         ReLU output that feeds both a concatenation and a pool
 * out is rounded to BF16 as the network stores it.  D, H, W even for ops 0
 * and 3; b, c used by op 3 only.
 */
gbsw_status unet_glue(int op, int nsamples, int D, int H, int W, int C, const float *a, const float *b,
                      const float *c, float *out, void *stream);

/*
 * The 1x1 head and the MSE loss: out[v] = hb + sum_c d1[v][c] hw[c]
 * (d1 nvox*16, rounded to BF16; hw 16, hb 1 FP32).  With target (nvox)
 * non-NULL also the backward pass of L = mean (out - target)^2:
 * *loss = L (FP64), g_hw[c] = sum_v dL/dout_v d1[v][c], *g_hb = sum_v
 * dL/dout_v, g_d1[v][c] = dL/dout_v hw[c] where d1[v][c] > 0 else 0
 * (rounded to BF16).  1 <= nvox <= 2^30.
 */
gbsw_status unet_head(long long nvox, const float *d1, const float *hw, const float *hb, const float *target,
                      float *out, float *g_hw, float *g_hb, float *g_d1, double *loss, void *stream);

typedef struct gbsw_unet gbsw_unet;

/* Number of FP32 parameters: for each 3x3x3 layer l1a (2->16), l1b (16->16),
 * l2a (16->32), l2b (32->32), l3a (32->64), l3b (64->32), l2c (64->16),
 * l1c (32->16) the weights w[27][cout][cin] then the bias[cout], followed
 * by the 1x1 head's 16 weights and its bias. */
int unet_num_params(void);

/* Create the network with He-normal weights drawn from `seed`. */
gbsw_status unet_create(unsigned long long seed, void *stream, gbsw_unet **out);

/* Copy all n = unet_num_params() parameters to / from host memory. */
gbsw_status unet_get_params(gbsw_unet *net, float *host, int n);
gbsw_status unet_set_params(gbsw_unet *net, const float *host, int n);

/*
 * Forward pass.  x: device, n*D*H*W*2 FP32 (channels last; for the warm
 * start the features of warm_start_features); y: device, n*D*H*W FP32.
 * D, H, W multiples of 4; each level (1, 1/2, 1/4) must meet the geometry
 * rule of unet_conv3d (e.g. 16x16x8, whose levels are 16x16, 8x8, 4x4
 * planes).  Synchronous.
 */
gbsw_status unet_forward(gbsw_unet *net, int n, int D, int H, int W, const float *x, float *y);

/* The same forward pass under the name of the boundary's inference call. */
gbsw_status unet_infer(gbsw_unet *net, int n, int D, int H, int W, const float *x, float *y);

/* MSE loss against target (device, n*D*H*W FP32) and the parameter
 * gradients (host array of unet_num_params(), or NULL), no update. */
gbsw_status unet_gradients(gbsw_unet *net, int n, int D, int H, int W, const float *x, const float *target,
                           float *grads_host, double *loss);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the MSE loss; *loss
 * (host, may be NULL) receives the loss before the update. */
gbsw_status unet_train_step(gbsw_unet *net, int n, int D, int H, int W, const float *x, const float *target,
                            float lr, double *loss);

void unet_destroy(gbsw_unet *net);

/*
 * Learned warm start for les_step (the "press" step of Sec. 6.3.1 keeps its
 * SOR; only the initial guess changes).  Before each solve the network runs
 * on the grid coarsened by a factor f, where its receptive field spans the
 * domain (the smooth modes that set the SOR iteration count are global):
 * the input is warm_start_features of the right-hand side b and the
 * previous pressure, and the prolongated, rescaled output is added to the
 * previous pressure (warm_start_apply).  SOR then runs to the same
 * tolerance, so the plain solve still decides the answer.
 * net = NULL restores the plain warm start (previous pressure).  The
 * context does not own the network; keep it alive while it is set.
 * GBSW_ERR_ARG if the network does not fit the coarse grid (see
 * les_set_warm_start_factor).
 */
gbsw_status les_set_warm_start(gbsw_les *les, gbsw_unet *net);

/* Coarsening factor f of the warm start: a power of two dividing nx, ny,
 * nz such that the coarse grid meets unet_forward's shape rule, or 0 for
 * the default (the largest such f <= 16; 16 on a 256 x 256 x 128 grid,
 * whose coarse grid is 16 x 16 x 8).  GBSW_ERR_ARG otherwise. */
gbsw_status les_set_warm_start_factor(gbsw_les *les, int f);

/*
 * Network input of the warm start, on caller-owned device arrays:
 *   p      device, nz*ny*nx FP64, the previous pressure (dense, x fastest)
 *   b      device, nz*ny*nx FP32, the right-hand side (divergence / dt)
 *   x      device, out: (nz/f)(ny/f)(nx/f) x 2 FP32, channels last:
 *          [r_c / rms(r_c), p_c / rms(p_c)], r_c and p_c the full-weighted
 *          restrictions (the adjoint of warm_start_apply's prolongation,
 *          divided by f^3) of r = b - A p and of p (A: the operator of
 *          poisson_solve)
 *   scale  host, out: s = (f dx)^2 rms(r_c), the unit of the network's output
 * f a power of two dividing nx, ny, nz.  Sums in FP64, fixed order.
 * Synchronous.  The training target for a converged pressure p_new is the
 * block mean of (p_new - p) / s.
 */
gbsw_status warm_start_features(int nx, int ny, int nz, double dx, int f, const double *p, const float *b,
                                float *x, double *scale, void *stream);

/*
 * p += scale * prolong(out): out device (nz/f)(ny/f)(nx/f) FP32, p device
 * nz*ny*nx FP64 (dense).  prolong is trilinear between coarse cell centres,
 * holding the end values at the inflow, ground and lid, with the ghost
 * past the outflow equal to minus the last value (p = 0 on that face) and
 * wrapping in y.  Synchronous.
 */
gbsw_status warm_start_apply(int nx, int ny, int nz, int f, const float *out, double scale, double *p,
                             void *stream);

/*
 * Volume reduction that allocates no memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc, such as applications whose own memory pool owns the whole
 * device, or latency-critical loops where an allocation (which may
 * synchronise the device) or an out-of-memory failure mid-run is not
 * acceptable.
 *
 * Computes what sw_volume computes, on caller-owned device fields:
 *   H, eta  device, ny rows of `pitch` floats (pitch >= nx), cell (i, j)
 *           at j*pitch + i; read only.
 *   out     device, 3 doubles written: dx*dy*sum(H + eta), the same over
 *           wet cells (H + eta > hmin, FP32 test), and the count of
 *           non-finite eta values.
 * Sizes: 1 <= nx, ny <= 1048576, otherwise GBSW_ERR_ARG; NULL pointers or
 * non-positive dx, dy are GBSW_ERR_ARG.  Asynchronous on `stream`; the
 * result is bitwise equal to sw_volume's for the same fields.
 *
 * The partial sums live in a fixed 24 KB array inside the library (one
 * per GPU, held until the process exits), so no call allocates anything.
 * The first call in a device's CUDA context looks up that array's device
 * address (a set-up done once per device with that device current, and
 * again if the device's context is destroyed and re-created); make that
 * first call before any stream capture.  All calls share the array and each call overwrites
 * it completely: calls whose kernels can overlap on the GPU (other streams
 * or host threads) race and must be serialised by the caller.
 */
gbsw_status sw_volume_noalloc(int nx, int ny, int pitch, double dx, double dy, double hmin,
                              const float *H, const float *eta, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GBSW_H */

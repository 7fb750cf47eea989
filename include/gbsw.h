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
 *    default stream.  Calls on one context are not thread-safe.
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
 * 0 = automatic, else 1..6. */
gbsw_status sw_set_blocking(gbsw_sw *sw, int steps_per_launch);

/* Release the context and its device memory.  NULL is ignored. */
void sw_destroy(gbsw_sw *sw);

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
 * The first call on a device looks up that array's device address (a
 * one-time set-up with that device current); make that first call before
 * any stream capture.  All calls share the array and each call overwrites
 * it completely: calls whose kernels can overlap on the GPU (other streams
 * or host threads) race and must be serialised by the caller.
 */
gbsw_status sw_volume_noalloc(int nx, int ny, int pitch, double dx, double dy, double hmin,
                              const float *H, const float *eta, double *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GBSW_H */

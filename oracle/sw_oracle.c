/*
 * FP64 CPU oracle of the 2-D shallow-water time step (the "2DSW" test case,
 * Sec. 6.2 of Vanderbauwhede & Davidson, arXiv:1711.04471).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code;
 * it exists so that tests, the smoke check and the timed CPU baseline can
 * compare the CUDA kernels against an obviously correct, slow reference.
 * It shares no source with the CUDA library.
 *
 * Sec. 6.2 describes the model as a time loop that calls a predictor ("dyn")
 * and a first-order Shapiro filter ("shapiro") and then updates the
 * velocity.  The paper prints no equations, so the discretisation below is
 * this project's reading of that structure (listed as readings in the
 * design notes):
 *
 *   staggered C-grid, interior cells i = 1..nx, j = 1..ny, one halo ring;
 *   eta, H at cell centres; u on the east face of cell (i,j) (i = 0..nx),
 *   v on the north face (j = 0..ny); faces on the closed walls are 0.
 *
 *   per step, every map reads the arrays of the start of the step:
 *   1  h = H + eta, wet = h > hmin (halo cells are dry).
 *   2  dyn/momentum: u' = u - g dt (eta_e - eta_c)/dx on interior faces,
 *      kept only if (wet_c and wet_e) or (wet_c and u' > 0) or
 *      (wet_e and u' < 0); otherwise 0.  Same for v' in y.
 *   3  dyn/continuity: upwind face fluxes F = max(u',0) h_c + min(u',0) h_e,
 *      eta* = eta - dt [ (F_e - F_w)/dx + (G_n - G_s)/dy ] on every cell.
 *   4  shapiro: on wet cells, eta+ = (1 - eps/4 sum_nb wet_nb) eta*_c
 *      + eps/4 sum_nb wet_nb eta*_nb; dry cells keep eta*.
 *   5  update: eta = eta+, u = u', v = v'.
 *
 * Arrays are (ny+2) x (nx+2) doubles, row-major, x fastest, index
 * j*(nx+2) + i.  Build with -O2 -ffp-contract=off so every operation rounds
 * as written.
 *
 * Threads: built with -fopenmp (the all-cores timing build), the outer loop
 * of each per-cell map runs in parallel.  Every cell's value is computed by
 * the same expression either way, and the volume sum stays serial, so both
 * builds give bitwise equal results.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j) ((size_t)(j) * (size_t)(nx + 2) + (size_t)(i))

typedef struct {
    int nx, ny;
    double dx, dy, dt, g, eps, hmin;
} oracle_sw_params;

/* Step 1: total depth and wet mask of the start of the step. */
static void sw_depth_and_mask(const oracle_sw_params *p, const double *H, const double *eta,
                              double *h, unsigned char *wet)
{
    const int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j <= ny + 1; ++j)
        for (int i = 0; i <= nx + 1; ++i) {
            int interior = (i >= 1 && i <= nx && j >= 1 && j <= ny);
            double hh = interior ? H[IDX(i, j)] + eta[IDX(i, j)] : 0.0;
            h[IDX(i, j)] = hh;
            wet[IDX(i, j)] = (unsigned char)(interior && hh > p->hmin);
        }
}

/* Face-mask rule shared by u and v: a is the cell behind the face (west or
 * south), b the cell ahead of it (east or north). */
static double sw_mask_face(double vel, unsigned char wet_a, unsigned char wet_b)
{
    if (wet_a && wet_b) return vel;
    if (wet_a && vel > 0.0) return vel;
    if (wet_b && vel < 0.0) return vel;
    return 0.0;
}

/* Step 2 ("dyn", momentum predictor). */
static void sw_dyn_momentum(const oracle_sw_params *p, const double *eta, const unsigned char *wet,
                            const double *u, const double *v, double *un, double *vn)
{
    const int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
    for (int j = 1; j <= ny; ++j)
        for (int i = 0; i <= nx; ++i) {
            double val = 0.0;
            if (i >= 1 && i <= nx - 1) {
                double pred = u[IDX(i, j)] - p->g * p->dt * (eta[IDX(i + 1, j)] - eta[IDX(i, j)]) / p->dx;
                val = sw_mask_face(pred, wet[IDX(i, j)], wet[IDX(i + 1, j)]);
            }
            un[IDX(i, j)] = val;
        }
#pragma omp parallel for schedule(static)
    for (int j = 0; j <= ny; ++j)
        for (int i = 1; i <= nx; ++i) {
            double val = 0.0;
            if (j >= 1 && j <= ny - 1) {
                double pred = v[IDX(i, j)] - p->g * p->dt * (eta[IDX(i, j + 1)] - eta[IDX(i, j)]) / p->dy;
                val = sw_mask_face(pred, wet[IDX(i, j)], wet[IDX(i, j + 1)]);
            }
            vn[IDX(i, j)] = val;
        }
}

/* Upwind volume flux through a face with velocity vel between cells a (behind) and b (ahead). */
static double sw_upwind_flux(double vel, double h_a, double h_b)
{
    double up = vel > 0.0 ? vel : 0.0;
    double dn = vel < 0.0 ? vel : 0.0;
    return up * h_a + dn * h_b;
}

/* Step 3 ("dyn", continuity). */
static void sw_dyn_continuity(const oracle_sw_params *p, const double *h, const double *un,
                              const double *vn, const double *eta, double *eta_star)
{
    const int nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
    for (int j = 1; j <= ny; ++j)
        for (int i = 1; i <= nx; ++i) {
            double fe = sw_upwind_flux(un[IDX(i, j)], h[IDX(i, j)], h[IDX(i + 1, j)]);
            double fw = sw_upwind_flux(un[IDX(i - 1, j)], h[IDX(i - 1, j)], h[IDX(i, j)]);
            double gn = sw_upwind_flux(vn[IDX(i, j)], h[IDX(i, j)], h[IDX(i, j + 1)]);
            double gs = sw_upwind_flux(vn[IDX(i, j - 1)], h[IDX(i, j - 1)], h[IDX(i, j)]);
            eta_star[IDX(i, j)] = eta[IDX(i, j)] - p->dt * ((fe - fw) / p->dx + (gn - gs) / p->dy);
        }
}

/* Step 4 ("shapiro"): masked 5-point first-order filter on wet cells. */
static void sw_shapiro(const oracle_sw_params *p, const unsigned char *wet, const double *eta_star,
                       double *eta_new)
{
    const int nx = p->nx, ny = p->ny;
    const double q = 0.25 * p->eps;
#pragma omp parallel for schedule(static)
    for (int j = 1; j <= ny; ++j)
        for (int i = 1; i <= nx; ++i) {
            if (!wet[IDX(i, j)]) {
                eta_new[IDX(i, j)] = eta_star[IDX(i, j)];
                continue;
            }
            const int ni[4] = {i + 1, i - 1, i, i};
            const int nj[4] = {j, j, j + 1, j - 1};
            double count = 0.0, sum = 0.0;
            for (int k = 0; k < 4; ++k)
                if (wet[IDX(ni[k], nj[k])]) {
                    count += 1.0;
                    sum += eta_star[IDX(ni[k], nj[k])];
                }
            eta_new[IDX(i, j)] = (1.0 - q * count) * eta_star[IDX(i, j)] + q * sum;
        }
}

/* Workspace for one run, allocated per call to keep the oracle reentrant. */
typedef struct {
    double *h, *un, *vn, *eta_star, *eta_new;
    unsigned char *wet;
} sw_work;

static int sw_work_alloc(sw_work *w, size_t n)
{
    w->h = calloc(n, sizeof(double));
    w->un = calloc(n, sizeof(double));
    w->vn = calloc(n, sizeof(double));
    w->eta_star = calloc(n, sizeof(double));
    w->eta_new = calloc(n, sizeof(double));
    w->wet = calloc(n, 1);
    return (w->h && w->un && w->vn && w->eta_star && w->eta_new && w->wet) ? 0 : -1;
}

static void sw_work_free(sw_work *w)
{
    free(w->h); free(w->un); free(w->vn); free(w->eta_star); free(w->eta_new); free(w->wet);
}

/*
 * Advance (eta, u, v) by nsteps.  H, eta, u, v are (ny+2) x (nx+2) arrays;
 * eta is read and written on interior cells, u and v on their faces.
 * If margin != NULL it receives min over all steps and interior cells of
 * |h - hmin| (the wet/dry margin certificate).  Returns 0, or -1 on
 * allocation failure.
 */
int oracle_sw_run(const oracle_sw_params *p, const double *H, double *eta, double *u, double *v,
                  int nsteps, double *margin)
{
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)(nx + 2) * (size_t)(ny + 2);
    sw_work w;
    if (sw_work_alloc(&w, n) != 0) {
        sw_work_free(&w);
        return -1;
    }
    double m = INFINITY;
    for (int s = 0; s < nsteps; ++s) {
        sw_depth_and_mask(p, H, eta, w.h, w.wet);
#pragma omp parallel for schedule(static) reduction(min : m)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                double d = fabs(w.h[IDX(i, j)] - p->hmin);
                if (d < m) m = d;
            }
        sw_dyn_momentum(p, eta, w.wet, u, v, w.un, w.vn);
        sw_dyn_continuity(p, w.h, w.un, w.vn, eta, w.eta_star);
        sw_shapiro(p, w.wet, w.eta_star, w.eta_new);
        /* Step 5: state update. */
#pragma omp parallel for schedule(static)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i)
                eta[IDX(i, j)] = w.eta_new[IDX(i, j)];
        memcpy(u, w.un, n * sizeof(double));
        memcpy(v, w.vn, n * sizeof(double));
    }
    /* The margin also covers the final state, which decides the last mask. */
    sw_depth_and_mask(p, H, eta, w.h, w.wet);
#pragma omp parallel for schedule(static) reduction(min : m)
    for (int j = 1; j <= ny; ++j)
        for (int i = 1; i <= nx; ++i) {
            double d = fabs(w.h[IDX(i, j)] - p->hmin);
            if (d < m) m = d;
        }
    if (margin) *margin = m;
    sw_work_free(&w);
    return 0;
}

/*
 * Total volume dx*dy*sum_interior (H + eta) and the volume held by wet
 * cells, in FP64 with a plain left-to-right sum.
 */
void oracle_sw_volume(const oracle_sw_params *p, const double *H, const double *eta,
                      double *volume, double *wet_volume)
{
    const int nx = p->nx, ny = p->ny;
    double s = 0.0, sw = 0.0;
    for (int j = 1; j <= ny; ++j)
        for (int i = 1; i <= nx; ++i) {
            double h = H[IDX(i, j)] + eta[IDX(i, j)];
            s += h;
            if (h > p->hmin) sw += h;
        }
    *volume = s * p->dx * p->dy;
    *wet_volume = sw * p->dx * p->dy;
}

/* Threads the parallel maps use (1 in the serial build); n > 0 sets it. */
int oracle_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

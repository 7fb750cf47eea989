/*
 * FP64 CPU oracle of the UFLES time step (Large Eddy Simulator for Urban
 * Flows, Sec. 6.3 of Vanderbauwhede & Davidson, arXiv:1711.04471).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the timed
 * CPU baseline, never by the product path; it shares no source with the
 * CUDA library.
 *
 * Sec. 6.3.1 lists the seven subroutines the main loop calls each step, in
 * this order: velnw (update velocity), bondv1 (boundary conditions: wind
 * profile, inflow, outflow), velfg (body force), feedbf (building effects,
 * Goldstein damping), les (viscosity, Smagorinsky model), adam
 * (Adams-Bashforth integration), press (Poisson equation for pressure by
 * SOR).  The paper gives no equations; the discretisation is this
 * project's reading (listed in the design notes):
 *
 *   grid: nx*ny*nz cells of size dx (isotropic), one ghost layer.
 *   u on east faces (i = 0..nx; 0 = inflow plane, nx = outflow plane),
 *   v on north faces (j = 1..ny, periodic in y), w on top faces
 *   (k = 0..nz; 0 = ground and nz = lid are 0), p and nu_t at centres.
 *
 *   velnw : u = u* - dt dp/dx on faces 1..nx (ghost p beyond the outflow
 *           plane = -p: p = 0 there), v likewise (periodic), w on 1..nz-1.
 *   bondv1: inflow face u = u_ref ln(z/z0)/ln(z_ref/z0); ghosts: v, w = 0
 *           at inflow (mirror with sign flip), zero gradient at outflow,
 *           periodic in y, no slip at the ground (mirror, sign flip),
 *           free slip at the lid (mirror).
 *   velfg : F = -div(u (x) u), flux form, 2nd-order central averages.
 *   feedbf: on faces touching a building cell, G += dt u and
 *           F += alpha G + beta u.
 *   les   : nu_t = (cs dx)^2 sqrt(2 S:S) at centres, F += div(2 (nu+nu_t) S)
 *           with nu_eff averaged to edges.
 *   adam  : u* = u + dt (1.5 F - 0.5 F_old) (Euler on the first step),
 *           F_old = F.
 *   press : b = div(u*)/dt; red-black SOR for A p = b, A the 7-point
 *           Laplacian with Neumann at inflow, ground and lid, Dirichlet
 *           p = 0 at the outflow face, periodic in y; stop when
 *           ||b - A p||_2 / ||b||_2 <= tol (checked every iteration).
 *
 * Arrays are (nz+2)*(ny+2)*(nx+2) doubles, x fastest.
 * Build with -O2 -ffp-contract=off.
 *
 * Threads: built with -fopenmp (the all-cores timing build), the outer loop
 * of each per-cell map runs in parallel, and the two colours of an SOR
 * iteration stay in order (cells of one colour read only the other
 * colour).  The residual norms are summed serially in the same cell order
 * in both builds (the OpenMP build first stores the per-cell terms), so
 * both builds give bitwise equal results.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;
    double dx, dt;
    double u_ref, z_ref, z0;
    double cs, nu, alpha, beta;
    double omega, tol;
    int max_iter;
} oracle_les_params;

#define NXP (P->nx + 2)
#define NYP (P->ny + 2)
#define ID(i, j, k) (((size_t)(k) * (size_t)NYP + (size_t)(j)) * (size_t)NXP + (size_t)(i))

/* Marker so the Python side knows the LES entry points exist. */
int oracle_les_declare_marker(void) { return 1; }

static double inflow_u(const oracle_les_params *P, int k)
{
    double z = ((double)k - 0.5) * P->dx;
    return P->u_ref * log(z / P->z0) / log(P->z_ref / P->z0);
}

/* ------------------------------------------------------------------ velnw */
void oracle_les_velnw(const oracle_les_params *P, const double *p, double *u, double *v, double *w)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const double c = P->dt / P->dx;
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                double pe = (i < nx) ? p[ID(i + 1, j, k)] : -p[ID(i, j, k)];
                u[ID(i, j, k)] -= c * (pe - p[ID(i, j, k)]);
                int jn = (j < ny) ? j + 1 : 1;
                v[ID(i, j, k)] -= c * (p[ID(i, jn, k)] - p[ID(i, j, k)]);
                if (k < nz) w[ID(i, j, k)] -= c * (p[ID(i, j, k + 1)] - p[ID(i, j, k)]);
            }
}

/* ----------------------------------------------------------------- bondv1 */
/* Inflow face values and the ghost layer of u, v, w (x, then y, then z). */
void oracle_les_bondv1(const oracle_les_params *P, double *u, double *v, double *w)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz;
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j) {
            u[ID(0, j, k)] = inflow_u(P, k);
            u[ID(nx + 1, j, k)] = u[ID(nx, j, k)];
            v[ID(0, j, k)] = -v[ID(1, j, k)];
            v[ID(nx + 1, j, k)] = v[ID(nx, j, k)];
            w[ID(0, j, k)] = -w[ID(1, j, k)];
            w[ID(nx + 1, j, k)] = w[ID(nx, j, k)];
        }
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= nz; ++k)
        for (int i = 0; i <= nx + 1; ++i) {
            u[ID(i, 0, k)] = u[ID(i, ny, k)];
            u[ID(i, ny + 1, k)] = u[ID(i, 1, k)];
            v[ID(i, 0, k)] = v[ID(i, ny, k)];
            v[ID(i, ny + 1, k)] = v[ID(i, 1, k)];
            w[ID(i, 0, k)] = w[ID(i, ny, k)];
            w[ID(i, ny + 1, k)] = w[ID(i, 1, k)];
        }
#pragma omp parallel for schedule(static)
    for (int j = 0; j <= ny + 1; ++j)
        for (int i = 0; i <= nx + 1; ++i) {
            u[ID(i, j, 0)] = -u[ID(i, j, 1)];
            v[ID(i, j, 0)] = -v[ID(i, j, 1)];
            w[ID(i, j, 0)] = 0.0;
            u[ID(i, j, nz + 1)] = u[ID(i, j, nz)];
            v[ID(i, j, nz + 1)] = v[ID(i, j, nz)];
            w[ID(i, j, nz)] = 0.0;
            w[ID(i, j, nz + 1)] = 0.0;
        }
}

/* ------------------------------------------------------------------ velfg */
/* F = -(advection) in flux form on u faces i=1..nx, v faces j=1..ny,
 * w faces k=1..nz-1 (other entries set to 0). */
void oracle_les_velfg(const oracle_les_params *P, const double *u, const double *v, const double *w,
                      double *fu, double *fv, double *fw)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const size_t n = (size_t)NXP * NYP * (nz + 2);
    memset(fu, 0, n * sizeof(double));
    memset(fv, 0, n * sizeof(double));
    memset(fw, 0, n * sizeof(double));
    const double r = 1.0 / P->dx;
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                /* u at face (i+1/2, j, k) */
                {
                    double ue = 0.5 * (u[ID(i, j, k)] + u[ID(i + 1, j, k)]);
                    double uw = 0.5 * (u[ID(i - 1, j, k)] + u[ID(i, j, k)]);
                    double un = 0.5 * (u[ID(i, j, k)] + u[ID(i, j + 1, k)]) * 0.5 * (v[ID(i, j, k)] + v[ID(i + 1, j, k)]);
                    double us = 0.5 * (u[ID(i, j - 1, k)] + u[ID(i, j, k)]) * 0.5 * (v[ID(i, j - 1, k)] + v[ID(i + 1, j - 1, k)]);
                    double ut = 0.5 * (u[ID(i, j, k)] + u[ID(i, j, k + 1)]) * 0.5 * (w[ID(i, j, k)] + w[ID(i + 1, j, k)]);
                    double ub = 0.5 * (u[ID(i, j, k - 1)] + u[ID(i, j, k)]) * 0.5 * (w[ID(i, j, k - 1)] + w[ID(i + 1, j, k - 1)]);
                    fu[ID(i, j, k)] = -r * ((ue * ue - uw * uw) + (un - us) + (ut - ub));
                }
                /* v at face (i, j+1/2, k) */
                {
                    double ve = 0.5 * (v[ID(i, j, k)] + v[ID(i + 1, j, k)]) * 0.5 * (u[ID(i, j, k)] + u[ID(i, j + 1, k)]);
                    double vw = 0.5 * (v[ID(i - 1, j, k)] + v[ID(i, j, k)]) * 0.5 * (u[ID(i - 1, j, k)] + u[ID(i - 1, j + 1, k)]);
                    double vn = 0.5 * (v[ID(i, j, k)] + v[ID(i, j + 1, k)]);
                    double vs = 0.5 * (v[ID(i, j - 1, k)] + v[ID(i, j, k)]);
                    double vt = 0.5 * (v[ID(i, j, k)] + v[ID(i, j, k + 1)]) * 0.5 * (w[ID(i, j, k)] + w[ID(i, j + 1, k)]);
                    double vb = 0.5 * (v[ID(i, j, k - 1)] + v[ID(i, j, k)]) * 0.5 * (w[ID(i, j, k - 1)] + w[ID(i, j + 1, k - 1)]);
                    fv[ID(i, j, k)] = -r * ((ve - vw) + (vn * vn - vs * vs) + (vt - vb));
                }
                /* w at face (i, j, k+1/2) */
                if (k < nz) {
                    double we = 0.5 * (w[ID(i, j, k)] + w[ID(i + 1, j, k)]) * 0.5 * (u[ID(i, j, k)] + u[ID(i, j, k + 1)]);
                    double ww = 0.5 * (w[ID(i - 1, j, k)] + w[ID(i, j, k)]) * 0.5 * (u[ID(i - 1, j, k)] + u[ID(i - 1, j, k + 1)]);
                    double wn = 0.5 * (w[ID(i, j, k)] + w[ID(i, j + 1, k)]) * 0.5 * (v[ID(i, j, k)] + v[ID(i, j, k + 1)]);
                    double ws = 0.5 * (w[ID(i, j - 1, k)] + w[ID(i, j, k)]) * 0.5 * (v[ID(i, j - 1, k)] + v[ID(i, j - 1, k + 1)]);
                    double wt = 0.5 * (w[ID(i, j, k)] + w[ID(i, j, k + 1)]);
                    double wb = 0.5 * (w[ID(i, j, k - 1)] + w[ID(i, j, k)]);
                    fw[ID(i, j, k)] = -r * ((we - ww) + (wn - ws) + (wt * wt - wb * wb));
                }
            }
}

/* ----------------------------------------------------------------- feedbf */
/* Faces touching a solid cell: G += dt u, F += alpha G + beta u. */
void oracle_les_feedbf(const oracle_les_params *P, const unsigned char *solid, const double *u, const double *v,
                       const double *w, double *gu, double *gv, double *gw, double *fu, double *fv, double *fw)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    /* solid is nz*ny*nx without ghosts */
#define SOL(i, j, k) (solid[((size_t)((k) - 1) * ny + (size_t)((j) - 1)) * nx + (size_t)((i) - 1)])
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                const int s = SOL(i, j, k);
                const int se = (i < nx) ? SOL(i + 1, j, k) : 0;
                const int sn = SOL(i, (j < ny) ? j + 1 : 1, k);
                const int st = (k < nz) ? SOL(i, j, k + 1) : 0;
                const size_t c = ID(i, j, k);
                if (s || se) {
                    gu[c] += P->dt * u[c];
                    fu[c] += P->alpha * gu[c] + P->beta * u[c];
                }
                if (s || sn) {
                    gv[c] += P->dt * v[c];
                    fv[c] += P->alpha * gv[c] + P->beta * v[c];
                }
                if (k < nz && (s || st)) {
                    gw[c] += P->dt * w[c];
                    fw[c] += P->alpha * gw[c] + P->beta * w[c];
                }
            }
#undef SOL
}

/* -------------------------------------------------------------------- les */
/* Strain-rate pieces at their natural points (see header). */
static double s12_edge(const oracle_les_params *P, const double *u, const double *v, int i, int j, int k)
{ /* edge (i+1/2, j+1/2, k) */
    return 0.5 * ((u[ID(i, j + 1, k)] - u[ID(i, j, k)]) + (v[ID(i + 1, j, k)] - v[ID(i, j, k)])) / P->dx;
}
static double s13_edge(const oracle_les_params *P, const double *u, const double *w, int i, int j, int k)
{ /* edge (i+1/2, j, k+1/2) */
    return 0.5 * ((u[ID(i, j, k + 1)] - u[ID(i, j, k)]) + (w[ID(i + 1, j, k)] - w[ID(i, j, k)])) / P->dx;
}
static double s23_edge(const oracle_les_params *P, const double *v, const double *w, int i, int j, int k)
{ /* edge (i, j+1/2, k+1/2) */
    return 0.5 * ((v[ID(i, j, k + 1)] - v[ID(i, j, k)]) + (w[ID(i, j + 1, k)] - w[ID(i, j, k)])) / P->dx;
}

/* Smagorinsky eddy viscosity at interior centres, ghosts filled by
 * zero gradient in x and z and periodicity in y. */
void oracle_les_nut(const oracle_les_params *P, const double *u, const double *v, const double *w, double *nut)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const double l2 = (P->cs * P->dx) * (P->cs * P->dx);
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                double s11 = (u[ID(i, j, k)] - u[ID(i - 1, j, k)]) / P->dx;
                double s22 = (v[ID(i, j, k)] - v[ID(i, j - 1, k)]) / P->dx;
                double s33 = (w[ID(i, j, k)] - w[ID(i, j, k - 1)]) / P->dx;
                double a12 = 0.0, a13 = 0.0, a23 = 0.0;
                for (int di = -1; di <= 0; ++di)
                    for (int dj = -1; dj <= 0; ++dj) {
                        double e = s12_edge(P, u, v, i + di, j + dj, k);
                        a12 += e * e;
                    }
                for (int di = -1; di <= 0; ++di)
                    for (int dk = -1; dk <= 0; ++dk) {
                        double e = s13_edge(P, u, w, i + di, j, k + dk);
                        a13 += e * e;
                    }
                for (int dj = -1; dj <= 0; ++dj)
                    for (int dk = -1; dk <= 0; ++dk) {
                        double e = s23_edge(P, v, w, i, j + dj, k + dk);
                        a23 += e * e;
                    }
                double ss = 2.0 * (s11 * s11 + s22 * s22 + s33 * s33) + 4.0 * 0.25 * (a12 + a13 + a23);
                nut[ID(i, j, k)] = l2 * sqrt(ss);
            }
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j) {
            nut[ID(0, j, k)] = nut[ID(1, j, k)];
            nut[ID(nx + 1, j, k)] = nut[ID(nx, j, k)];
        }
    for (int k = 1; k <= nz; ++k)
        for (int i = 0; i <= nx + 1; ++i) {
            nut[ID(i, 0, k)] = nut[ID(i, ny, k)];
            nut[ID(i, ny + 1, k)] = nut[ID(i, 1, k)];
        }
    for (int j = 0; j <= ny + 1; ++j)
        for (int i = 0; i <= nx + 1; ++i) {
            nut[ID(i, j, 0)] = nut[ID(i, j, 1)];
            nut[ID(i, j, nz + 1)] = nut[ID(i, j, nz)];
        }
}

/* F += div(2 nu_eff S) on the faces velfg fills; nut from oracle_les_nut. */
void oracle_les_visc(const oracle_les_params *P, const double *u, const double *v, const double *w,
                     const double *nut, double *fu, double *fv, double *fw)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const double r = 1.0 / P->dx, nu = P->nu;
#define NE(i, j, k) (nu + nut[ID(i, j, k)])
#define NU_XY(i, j, k) (0.25 * (NE(i, j, k) + NE(i + 1, j, k) + NE(i, j + 1, k) + NE(i + 1, j + 1, k)))
#define NU_XZ(i, j, k) (0.25 * (NE(i, j, k) + NE(i + 1, j, k) + NE(i, j, k + 1) + NE(i + 1, j, k + 1)))
#define NU_YZ(i, j, k) (0.25 * (NE(i, j, k) + NE(i, j + 1, k) + NE(i, j, k + 1) + NE(i, j + 1, k + 1)))
#define T11(i, j, k) (2.0 * NE(i, j, k) * (u[ID(i, j, k)] - u[ID(i - 1, j, k)]) * r)
#define T22(i, j, k) (2.0 * NE(i, j, k) * (v[ID(i, j, k)] - v[ID(i, j - 1, k)]) * r)
#define T33(i, j, k) (2.0 * NE(i, j, k) * (w[ID(i, j, k)] - w[ID(i, j, k - 1)]) * r)
#define T12(i, j, k) (2.0 * NU_XY(i, j, k) * s12_edge(P, u, v, i, j, k))
#define T13(i, j, k) (2.0 * NU_XZ(i, j, k) * s13_edge(P, u, w, i, j, k))
#define T23(i, j, k) (2.0 * NU_YZ(i, j, k) * s23_edge(P, v, w, i, j, k))
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                const size_t c = ID(i, j, k);
                fu[c] += r * ((T11(i + 1, j, k) - T11(i, j, k)) + (T12(i, j, k) - T12(i, j - 1, k)) +
                              (T13(i, j, k) - T13(i, j, k - 1)));
                fv[c] += r * ((T12(i, j, k) - T12(i - 1, j, k)) + (T22(i, j + 1, k) - T22(i, j, k)) +
                              (T23(i, j, k) - T23(i, j, k - 1)));
                if (k < nz)
                    fw[c] += r * ((T13(i, j, k) - T13(i - 1, j, k)) + (T23(i, j, k) - T23(i, j - 1, k)) +
                                  (T33(i, j, k + 1) - T33(i, j, k)));
            }
#undef NE
#undef NU_XY
#undef NU_XZ
#undef NU_YZ
#undef T11
#undef T22
#undef T33
#undef T12
#undef T13
#undef T23
}

/* ------------------------------------------------------------------- adam */
void oracle_les_adam(const oracle_les_params *P, int first, double *u, double *v, double *w, const double *fu,
                     const double *fv, const double *fw, double *fuo, double *fvo, double *fwo)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const double dt = P->dt;
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                const size_t c = ID(i, j, k);
                if (first) {
                    u[c] += dt * fu[c];
                    v[c] += dt * fv[c];
                    if (k < nz) w[c] += dt * fw[c];
                } else {
                    u[c] += dt * (1.5 * fu[c] - 0.5 * fuo[c]);
                    v[c] += dt * (1.5 * fv[c] - 0.5 * fvo[c]);
                    if (k < nz) w[c] += dt * (1.5 * fw[c] - 0.5 * fwo[c]);
                }
                fuo[c] = fu[c];
                fvo[c] = fv[c];
                fwo[c] = (k < nz) ? fw[c] : 0.0;
            }
}

/* ------------------------------------------------------------------ press */
/* b = div(u*)/dt at interior centres (v at j = 0 is the periodic image). */
void oracle_les_rhs(const oracle_les_params *P, const double *u, const double *v, const double *w, double *b)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const double c = 1.0 / (P->dx * P->dt);
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 1; i <= nx; ++i) {
                double vs = v[ID(i, (j > 1) ? j - 1 : ny, k)];
                b[ID(i, j, k)] = c * ((u[ID(i, j, k)] - u[ID(i - 1, j, k)]) + (v[ID(i, j, k)] - vs) +
                                      (w[ID(i, j, k)] - w[ID(i, j, k - 1)]));
            }
}

/* Neighbour sum and diagonal of the pressure operator at cell (i,j,k):
 * (A p)_c = (sum - diag * p_c) / dx^2. */
static void les_stencil(const oracle_les_params *P, const double *p, int i, int j, int k, double *sum, double *diag)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    double s = 0.0, d = 6.0;
    if (i > 1) s += p[ID(i - 1, j, k)]; else d -= 1.0;      /* Neumann at inflow */
    if (i < nx) s += p[ID(i + 1, j, k)]; else d += 1.0;     /* Dirichlet at outflow */
    s += p[ID(i, (j > 1) ? j - 1 : ny, k)];                 /* periodic in y */
    s += p[ID(i, (j < ny) ? j + 1 : 1, k)];
    if (k > 1) s += p[ID(i, j, k - 1)]; else d -= 1.0;      /* Neumann at ground */
    if (k < nz) s += p[ID(i, j, k + 1)]; else d -= 1.0;     /* Neumann at lid */
    *sum = s;
    *diag = d;
}

void oracle_les_apply_A(const oracle_les_params *P, const double *p, double *Ap)
{
    const double r2 = 1.0 / (P->dx * P->dx);
#pragma omp parallel for schedule(static)
    for (int k = 1; k <= P->nz; ++k)
        for (int j = 1; j <= P->ny; ++j)
            for (int i = 1; i <= P->nx; ++i) {
                double s, d;
                les_stencil(P, p, i, j, k, &s, &d);
                Ap[ID(i, j, k)] = (s - d * p[ID(i, j, k)]) * r2;
            }
}

/* Residual of cell (i,j,k): b - A p. */
static double les_res_cell(const oracle_les_params *P, const double *b, const double *p, double r2, int i, int j,
                           int k)
{
    double s, d;
    les_stencil(P, p, i, j, k, &s, &d);
    return b[ID(i, j, k)] - (s - d * p[ID(i, j, k)]) * r2;
}

/* ||b - A p||_2 / ||b||_2 over interior cells (0 if ||b|| == 0); the sums
 * run over the cells in (k, j, i) order.  work: NULL, or (OpenMP build)
 * 2 nx ny nz doubles for the per-cell terms, formed in parallel. */
static double les_residual_w(const oracle_les_params *P, const double *b, const double *p, double *work)
{
    const double r2 = 1.0 / (P->dx * P->dx);
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    double rr = 0.0, bb = 0.0;
    if (work) {
        const size_t nc = (size_t)nx * ny * nz;
#pragma omp parallel for schedule(static)
        for (int k = 1; k <= nz; ++k)
            for (int j = 1; j <= ny; ++j)
                for (int i = 1; i <= nx; ++i) {
                    const size_t q = ((size_t)(k - 1) * ny + (j - 1)) * nx + (i - 1);
                    const double res = les_res_cell(P, b, p, r2, i, j, k);
                    work[q] = res * res;
                    work[nc + q] = b[ID(i, j, k)] * b[ID(i, j, k)];
                }
        for (size_t q = 0; q < nc; ++q) {
            rr += work[q];
            bb += work[nc + q];
        }
    } else {
        for (int k = 1; k <= nz; ++k)
            for (int j = 1; j <= ny; ++j)
                for (int i = 1; i <= nx; ++i) {
                    const double res = les_res_cell(P, b, p, r2, i, j, k);
                    rr += res * res;
                    bb += b[ID(i, j, k)] * b[ID(i, j, k)];
                }
    }
    return bb > 0.0 ? sqrt(rr / bb) : 0.0;
}

/* Scratch for the per-cell residual terms in the OpenMP build (NULL in the
 * serial build, or if the allocation fails: the serial sum is then used). */
static double *les_residual_work(const oracle_les_params *P)
{
#ifdef _OPENMP
    return (double *)malloc(2 * (size_t)P->nx * P->ny * P->nz * sizeof(double));
#else
    (void)P;
    return NULL;
#endif
}

double oracle_les_residual(const oracle_les_params *P, const double *b, const double *p)
{
    double *work = les_residual_work(P);
    const double rho = les_residual_w(P, b, p, work);
    free(work);
    return rho;
}

/* One red-black SOR iteration: cells with (i+j+k) even first, then odd. */
static void les_sor_sweep(const oracle_les_params *P, const double *b, double *p, double omega)
{
    const double h2 = P->dx * P->dx;
    for (int colour = 0; colour < 2; ++colour)
#pragma omp parallel for schedule(static)
        for (int k = 1; k <= P->nz; ++k)
            for (int j = 1; j <= P->ny; ++j)
                for (int i = 1; i <= P->nx; ++i) {
                    if (((i + j + k) & 1) != colour) continue;
                    double s, d;
                    les_stencil(P, p, i, j, k, &s, &d);
                    double gs = (s - h2 * b[ID(i, j, k)]) / d;
                    p[ID(i, j, k)] += omega * (gs - p[ID(i, j, k)]);
                }
}

/* SOR from the guess in p until the relative residual <= tol or max_iter
 * iterations.  Returns 0 if converged, 1 otherwise. */
int oracle_les_sor(const oracle_les_params *P, const double *b, double *p, double omega, double tol,
                   int max_iter, int *iters, double *rel_res)
{
    double *work = les_residual_work(P);
    double rho = les_residual_w(P, b, p, work);
    int it = 0;
    while (rho > tol && it < max_iter) {
        les_sor_sweep(P, b, p, omega);
        ++it;
        rho = les_residual_w(P, b, p, work);
    }
    free(work);
    *iters = it;
    *rel_res = rho;
    return rho <= tol ? 0 : 1;
}

/* ------------------------------------------------------------- full step */
typedef struct {
    double *u, *v, *w, *p;          /* u, v, w hold u* between steps */
    double *fuo, *fvo, *fwo;        /* previous tendencies */
    double *gu, *gv, *gw;           /* Goldstein time integrals */
    double *fu, *fv, *fw, *nut, *b; /* work */
    int step;                       /* steps taken so far */
} oracle_les_state;

/* Initial state: u* = inflow profile on every x-face (0 on faces that touch
 * a building), v* = w* = 0, p = 0. */
void oracle_les_init(const oracle_les_params *P, const unsigned char *solid, oracle_les_state *S)
{
    const int nx = P->nx, ny = P->ny, nz = P->nz;
    const size_t n = (size_t)NXP * NYP * (nz + 2);
    double *arrs[] = {S->u, S->v, S->w, S->p, S->fuo, S->fvo, S->fwo, S->gu, S->gv, S->gw, S->fu, S->fv, S->fw,
                      S->nut, S->b};
    for (size_t a = 0; a < sizeof(arrs) / sizeof(arrs[0]); ++a) memset(arrs[a], 0, n * sizeof(double));
    for (int k = 1; k <= nz; ++k)
        for (int j = 1; j <= ny; ++j)
            for (int i = 0; i <= nx; ++i) {
                int s = (i >= 1) ? solid[((size_t)(k - 1) * ny + (j - 1)) * nx + (i - 1)] : 0;
                int se = (i < nx) ? solid[((size_t)(k - 1) * ny + (j - 1)) * nx + i] : 0;
                S->u[ID(i, j, k)] = (s || se) ? 0.0 : inflow_u(P, k);
            }
    S->step = 0;
}

/* One UFLES step in the paper's subroutine order.  Returns the SOR status
 * (0 converged, 1 not) and the iteration count / final residual. */
int oracle_les_step(const oracle_les_params *P, const unsigned char *solid, oracle_les_state *S, int *iters,
                    double *rel_res)
{
    oracle_les_velnw(P, S->p, S->u, S->v, S->w);
    oracle_les_bondv1(P, S->u, S->v, S->w);
    oracle_les_velfg(P, S->u, S->v, S->w, S->fu, S->fv, S->fw);
    oracle_les_feedbf(P, solid, S->u, S->v, S->w, S->gu, S->gv, S->gw, S->fu, S->fv, S->fw);
    oracle_les_nut(P, S->u, S->v, S->w, S->nut);
    oracle_les_visc(P, S->u, S->v, S->w, S->nut, S->fu, S->fv, S->fw);
    oracle_les_adam(P, S->step == 0, S->u, S->v, S->w, S->fu, S->fv, S->fw, S->fuo, S->fvo, S->fwo);
    oracle_les_rhs(P, S->u, S->v, S->w, S->b);
    S->step += 1;
    return oracle_les_sor(P, S->b, S->p, P->omega, P->tol, P->max_iter, iters, rel_res);
}

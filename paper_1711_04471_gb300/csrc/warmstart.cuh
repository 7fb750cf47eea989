// Grid transfers of the learned warm start (warmstart.cu).
#pragma once

#include "common.cuh"

namespace gbsw {

// A field of nx*ny*nz interior cells; cell (i, j, k), 1-based, sits at
// off + (k-1)*sz + (j-1)*sy + (i-1).  The LES padded layout has
// off = plane + pitch + 1, sy = pitch, sz = plane; a dense array off = 0.
struct WsGrid {
    int nx, ny, nz;
    long long sy, sz, off;
    long long extent;  // elements of each field (the bounds-checked build tests indices against it)
};

// f a power of two (<= 64) dividing nx, ny and nz.
bool ws_factor_ok(int nx, int ny, int nz, int f);

// Doubles of scratch that launch_ws_restrict needs.
size_t ws_scratch_doubles(int nx, int ny, int nz, int f);

// rc, pc: (nz/f)(ny/f)(nx/f) FP64 full-weighted restrictions of b - A p and
// of p (prolong^T / f^3).
gbsw_status launch_ws_restrict(const float *b, const double *p, const WsGrid &g, double dx, int f, double *scratch,
                               double *rc, double *pc, cudaStream_t s);
// xin (nc x 2 FP32) and *scale = hc2 * rms(rc) (device).
gbsw_status launch_ws_prepare(const double *rc, const double *pc, long long nc, double hc2, float *xin,
                              double *scale, cudaStream_t s);
// p += *scale * prolong(out), out dense (nz/f)(ny/f)(nx/f) FP32.
gbsw_status launch_ws_prolong(const float *out, const WsGrid &g, int f, const double *scale, double *p,
                              cudaStream_t s);

}  // namespace gbsw

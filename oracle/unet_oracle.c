/*
 * FP64 CPU oracle of the operators of the 3-D convolutional U-Net used as a
 * learned warm start for the pressure solve (the paper's "press", Sec. 6.3.1
 * of arXiv:1711.04471, solves the Poisson equation by SOR; the network only
 * proposes the starting guess, SOR still decides the answer).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests, the smoke check and the CPU
 * baseline, never by the product path; shares no source with the CUDA
 * library.
 *
 * Tensors are channels-last volumes of one sample: x[((z*H + y)*W + x)*C + c].
 * Convolution weights are w[tap][co][ci] with tap = (dz+1)*9 + (dy+1)*3 +
 * (dx+1) for offsets dz, dy, dx in {-1, 0, 1}; zero padding of one cell.
 *   conv:      y[v, co] = b[co] + sum_tap sum_ci w[tap][co][ci] x[v + off(tap), ci]
 *   bwd_data:  dx[v, ci] = sum_tap sum_co w[tap][co][ci] dy[v - off(tap), co]
 *   bwd_weight: dw[tap][co][ci] = sum_v dy[v, co] x[v + off(tap), ci], db[co] = sum_v dy[v, co]
 *   pool:      2x2x2 average;  upsample: 2x nearest neighbour.
 * Every sum is a plain loop in a fixed order.
 */
#include <stddef.h>
#include <string.h>

int oracle_unet_declare_marker(void) { return 2; }

static size_t vox(int z, int y, int x, int H, int W) { return ((size_t)z * H + y) * W + x; }

void oracle_conv3d_fwd(int D, int H, int W, int Cin, int Cout, const double *x, const double *w, const double *b,
                       double *y)
{
    for (int z = 0; z < D; ++z)
        for (int yy = 0; yy < H; ++yy)
            for (int xx = 0; xx < W; ++xx) {
                double *out = y + vox(z, yy, xx, H, W) * Cout;
                for (int co = 0; co < Cout; ++co) out[co] = b ? b[co] : 0.0;
                for (int tap = 0; tap < 27; ++tap) {
                    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                    const int sz = z + dz, sy = yy + dy, sx = xx + dx;
                    if (sz < 0 || sz >= D || sy < 0 || sy >= H || sx < 0 || sx >= W) continue;
                    const double *in = x + vox(sz, sy, sx, H, W) * Cin;
                    for (int co = 0; co < Cout; ++co) {
                        const double *wr = w + ((size_t)tap * Cout + co) * Cin;
                        double s = 0.0;
                        for (int ci = 0; ci < Cin; ++ci) s += wr[ci] * in[ci];
                        out[co] += s;
                    }
                }
            }
}

void oracle_conv3d_bwd_data(int D, int H, int W, int Cin, int Cout, const double *dy, const double *w, double *dx)
{
    memset(dx, 0, (size_t)D * H * W * Cin * sizeof(double));
    for (int z = 0; z < D; ++z)
        for (int yy = 0; yy < H; ++yy)
            for (int xx = 0; xx < W; ++xx) {
                const double *g = dy + vox(z, yy, xx, H, W) * Cout;
                for (int tap = 0; tap < 27; ++tap) {
                    const int dz = tap / 9 - 1, dyy = (tap / 3) % 3 - 1, dxx = tap % 3 - 1;
                    const int sz = z + dz, sy = yy + dyy, sx = xx + dxx;
                    if (sz < 0 || sz >= D || sy < 0 || sy >= H || sx < 0 || sx >= W) continue;
                    double *o = dx + vox(sz, sy, sx, H, W) * Cin;
                    for (int co = 0; co < Cout; ++co) {
                        const double *wr = w + ((size_t)tap * Cout + co) * Cin;
                        for (int ci = 0; ci < Cin; ++ci) o[ci] += wr[ci] * g[co];
                    }
                }
            }
}

void oracle_conv3d_bwd_weight(int D, int H, int W, int Cin, int Cout, const double *x, const double *dy,
                              double *dw, double *db)
{
    memset(dw, 0, (size_t)27 * Cout * Cin * sizeof(double));
    if (db) memset(db, 0, (size_t)Cout * sizeof(double));
    for (int z = 0; z < D; ++z)
        for (int yy = 0; yy < H; ++yy)
            for (int xx = 0; xx < W; ++xx) {
                const double *g = dy + vox(z, yy, xx, H, W) * Cout;
                if (db)
                    for (int co = 0; co < Cout; ++co) db[co] += g[co];
                for (int tap = 0; tap < 27; ++tap) {
                    const int dz = tap / 9 - 1, dyy = (tap / 3) % 3 - 1, dxx = tap % 3 - 1;
                    const int sz = z + dz, sy = yy + dyy, sx = xx + dxx;
                    if (sz < 0 || sz >= D || sy < 0 || sy >= H || sx < 0 || sx >= W) continue;
                    const double *in = x + vox(sz, sy, sx, H, W) * Cin;
                    for (int co = 0; co < Cout; ++co) {
                        double *dwr = dw + ((size_t)tap * Cout + co) * Cin;
                        for (int ci = 0; ci < Cin; ++ci) dwr[ci] += g[co] * in[ci];
                    }
                }
            }
}

/* y (D/2, H/2, W/2, C) = mean over each 2x2x2 block of x (D, H, W, C). */
void oracle_avgpool2_fwd(int D, int H, int W, int C, const double *x, double *y)
{
    const int d = D / 2, h = H / 2, w = W / 2;
    for (int z = 0; z < d; ++z)
        for (int yy = 0; yy < h; ++yy)
            for (int xx = 0; xx < w; ++xx)
                for (int c = 0; c < C; ++c) {
                    double s = 0.0;
                    for (int k = 0; k < 8; ++k)
                        s += x[vox(2 * z + (k >> 2), 2 * yy + ((k >> 1) & 1), 2 * xx + (k & 1), H, W) * C + c];
                    y[vox(z, yy, xx, h, w) * C + c] = s / 8.0;
                }
}

void oracle_avgpool2_bwd(int D, int H, int W, int C, const double *dy, double *dx)
{
    const int h = H / 2, w = W / 2;
    for (int z = 0; z < D; ++z)
        for (int yy = 0; yy < H; ++yy)
            for (int xx = 0; xx < W; ++xx)
                for (int c = 0; c < C; ++c)
                    dx[vox(z, yy, xx, H, W) * C + c] = dy[vox(z / 2, yy / 2, xx / 2, h, w) * C + c] / 8.0;
}

/* y (2D, 2H, 2W, C): each cell copied to its 2x2x2 block (D, H, W = input). */
void oracle_upsample2_fwd(int D, int H, int W, int C, const double *x, double *y)
{
    for (int z = 0; z < 2 * D; ++z)
        for (int yy = 0; yy < 2 * H; ++yy)
            for (int xx = 0; xx < 2 * W; ++xx)
                for (int c = 0; c < C; ++c)
                    y[vox(z, yy, xx, 2 * H, 2 * W) * C + c] = x[vox(z / 2, yy / 2, xx / 2, H, W) * C + c];
}

void oracle_upsample2_bwd(int D, int H, int W, int C, const double *dy, double *dx)
{
    memset(dx, 0, (size_t)D * H * W * C * sizeof(double));
    for (int z = 0; z < 2 * D; ++z)
        for (int yy = 0; yy < 2 * H; ++yy)
            for (int xx = 0; xx < 2 * W; ++xx)
                for (int c = 0; c < C; ++c)
                    dx[vox(z / 2, yy / 2, xx / 2, H, W) * C + c] += dy[vox(z, yy, xx, 2 * H, 2 * W) * C + c];
}

// Launch wrappers of the U-Net glue kernels (unet_ops.cu); C8-blocked
// tensors are addressed by (pointer, channel groups in the tensor, first
// group used).
#pragma once

#include "unet_internal.cuh"

namespace gbsw {

// Interior of an LES padded field: (nz+2) x (ny+2) x pitch, cell (i,j,k) at
// k*plane + j*pitch + i.
struct PadDims {
    int nx, ny, nz, pitch;
    long long plane;
};

using bf16 = __nv_bfloat16;

// db[co] += sum over the nvox voxels of g[v, co] (C8-blocked, C channels from group g_cg0).
gbsw_status launch_bias_grad(const bf16 *g, int g_cg_total, int g_cg0, long long nvox, int H, int W, int C,
                             float *db, cudaStream_t s);
gbsw_status launch_pool(const bf16 *x, int x_cg_total, int x_cg0, int NZ, int H, int W, int C, bf16 *y, int y_cg_total,
                        int y_cg0, cudaStream_t s);
gbsw_status launch_upsample(const bf16 *x, int x_cg_total, int x_cg0, int NZ, int H, int W, int C, bf16 *y,
                            int y_cg_total, int y_cg0, cudaStream_t s);
gbsw_status launch_upsample_bwd(const bf16 *x, int x_cg_total, int x_cg0, int NZ, int H, int W, int C, bf16 *y,
                                int y_cg_total, int y_cg0, cudaStream_t s);
gbsw_status launch_pool_bwd_add_mask(const bf16 *from_cat, int c_cg_total, int c_cg0, const bf16 *from_pool,
                                     int p_cg_total, int p_cg0, const bf16 *act, int a_cg_total, int a_cg0, int NZ,
                                     int H, int W, int C, bf16 *out, int o_cg_total, int o_cg0, cudaStream_t s);
gbsw_status launch_head_fwd(const bf16 *d1, int cg_total, int cg0, long long nvox, int H, int W, const float *hw,
                            const float *hb, float *out, cudaStream_t s);
gbsw_status launch_head_bwd(const bf16 *d1, int cg_total, int cg0, long long nvox, int H, int W, const float *out,
                            const float *target, const float *hw, float *g_hw, float *g_hb, bf16 *g_d1, double *loss,
                            cudaStream_t s);
gbsw_status launch_adam(float *p, const float *g, float *m, float *v, int n, float lr, int step, cudaStream_t s);
// True if a (1, D, H, W) input fits the network: D, H, W multiples of 4 and
// every level within the tile geometry of the tcgen05 convolution.
bool unet_shape_ok(int D, int H, int W);

// LES hook: p += the network's pressure increment for right-hand side b
// and previous pressure p (padded LES layout), the network run on the grid
// coarsened by f (warmstart.cu), on stream s.  scratch: device, at least
// ws_scratch_doubles(nx, ny, nz, f) doubles.
gbsw_status unet_warm_start(gbsw_unet *u, const float *b, double *p, const PadDims &pd, double dx, int f,
                            double *scratch, cudaStream_t s);

}  // namespace gbsw

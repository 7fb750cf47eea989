// Internal interfaces between the U-Net translation units (not part of the ABI).
#pragma once

#include "unet_conv.cuh"

namespace gbsw {

// Arguments of one tcgen05 convolution launch.
struct ConvCall {
    CUtensorMap xmap;               // input, C8-blocked BF16 (all channel groups)
    const __nv_bfloat16 *wpack;     // packed weights [27][Cin/8][Cout][8]
    const float *bias;              // EPI_BIAS_RELU
    __nv_bfloat16 *y;               // C8-blocked output (may be NULL)
    float *y_f32;                   // dense (zn, y, x, Cout) FP32 output (may be NULL)
    const __nv_bfloat16 *mask;      // EPI_MASK
    ConvGeom geom;
    int epi;
    int *status;                    // device status word
};

gbsw_status conv_geometry(int NZ, int D, int H, int W, ConvGeom *g);
gbsw_status conv_tensor_map(const __nv_bfloat16 *base, const ConvGeom &g, int cg_total, CUtensorMap *map);
gbsw_status launch_conv(int cin, int cout, const ConvCall &c, cudaStream_t s);
gbsw_status launch_wgrad_tc(int cin, int cout, const WgradCall &c, cudaStream_t s);
gbsw_status pack_weights(const float *w, int cin, int cout, int flip, __nv_bfloat16 *pack, cudaStream_t s);
// As pack_weights from weights [27][cout][cin_src], input channels
// cin_src .. cin-1 packed as zeros (forward packs only).
gbsw_status pack_weights_padded(const float *w, int cin_src, int cin, int cout, int flip, __nv_bfloat16 *pack,
                                cudaStream_t s);
gbsw_status to_blocked(const float *src, int NZ, int H, int W, int C, __nv_bfloat16 *dst, int cg_total, int cg0,
                       cudaStream_t s);
gbsw_status from_blocked(const __nv_bfloat16 *src, int NZ, int H, int W, int C, int cg_total, int cg0, float *dst,
                         cudaStream_t s);

}  // namespace gbsw

// Operator-level entry points of the warm-start U-Net's kernels (see
// include/gbsw.h): each takes dense FP32 device tensors (n, D, H, W, C),
// C fastest, converts them to the kernels' C8-blocked BF16 layout
// (rounding to nearest even), runs exactly the kernel the network runs,
// and converts the result back, so that tests can compare every operator
// with the FP64 oracle on its own.
#include <vector>

#include "unet_ops.cuh"

using namespace gbsw;

namespace {

// Device scratch freed when the call returns.
struct Scratch {
    std::vector<void *> ptrs;
    ~Scratch()
    {
        for (void *p : ptrs) cudaFree(p);
    }
    template <typename T>
    gbsw_status get(T **p, size_t n)
    {
        GBSW_CUDA_TRY(cudaMalloc((void **)p, n * sizeof(T)));
        ptrs.push_back(*p);
        return GBSW_OK;
    }
};

#define CHK(x)                          \
    do {                                \
        gbsw_status _s = (x);           \
        if (_s != GBSW_OK) return _s;   \
    } while (0)

gbsw_status finish(int *status, cudaStream_t s)
{
    int h = 0;
    GBSW_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    GBSW_CUDA_TRY(cudaStreamSynchronize(s));
    return dev_status_to_gbsw(h);
}

bool pair_ok(int a, int b)
{
    const int ok[][2] = {{16, 16}, {16, 32}, {16, 64}, {32, 16}, {32, 32}, {32, 64}, {64, 16}, {64, 32}};
    for (const auto &p : ok)
        if (p[0] == a && p[1] == b) return true;
    return false;
}

}  // namespace

extern "C" gbsw_status unet_conv3d(int nsamples, int D, int H, int W, int cin, int cout, const float *x,
                                   const float *w, const float *bias, int epilogue, const float *mask, float *y,
                                   void *stream)
{
    const int cin_k = cin == 2 ? 16 : cin;  // two input channels run zero-padded to 16, as the first layer does
    if (!x || !w || !y || nsamples < 1 || !pair_ok(cin_k, cout) || epilogue < 0 || epilogue > 2) return GBSW_ERR_ARG;
    if (epilogue == EPI_BIAS_RELU && !bias) return GBSW_ERR_ARG;
    if (epilogue == EPI_MASK && !mask) return GBSW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ConvGeom g;
    CHK(conv_geometry(nsamples * D, D, H, W, &g));
    const size_t nv = (size_t)nsamples * D * H * W;
    Scratch sc;
    bf16 *xb = nullptr, *wp = nullptr, *mb = nullptr;
    int *status = nullptr;
    CHK(sc.get(&xb, nv * cin_k));
    CHK(sc.get(&wp, (size_t)27 * cin_k * cout));
    CHK(sc.get(&status, 1));
    GBSW_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    if (cin_k != cin) GBSW_CUDA_TRY(cudaMemsetAsync(xb, 0, nv * cin_k * sizeof(bf16), s));
    if (epilogue == EPI_MASK) {
        CHK(sc.get(&mb, nv * cout));
        CHK(to_blocked(mask, g.NZ, H, W, cout, mb, cout / 8, 0, s));
    }
    CHK(to_blocked(x, g.NZ, H, W, cin, xb, cin_k / 8, 0, s));
    CHK(pack_weights_padded(w, cin, cin_k, cout, 0, wp, s));
    ConvCall c{};
    CHK(conv_tensor_map(xb, g, cin_k / 8, &c.xmap));
    g.mask_cg_total = cout / 8;
    c.geom = g;
    c.wpack = wp;
    c.bias = bias;
    c.y_f32 = y;
    c.mask = mb;
    c.epi = epilogue;
    c.status = status;
    CHK(launch_conv(cin_k, cout, c, s));
    return finish(status, s);
}

extern "C" gbsw_status unet_conv3d_bwd_data(int nsamples, int D, int H, int W, int cin, int cout, const float *gy,
                                            const float *w, const float *mask, float *gx, void *stream)
{
    if (!gy || !w || !gx || nsamples < 1 || !pair_ok(cout, cin)) return GBSW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ConvGeom g;
    CHK(conv_geometry(nsamples * D, D, H, W, &g));
    const size_t nv = (size_t)nsamples * D * H * W;
    Scratch sc;
    bf16 *gyb = nullptr, *wp = nullptr, *mb = nullptr;
    int *status = nullptr;
    CHK(sc.get(&gyb, nv * cout));
    CHK(sc.get(&wp, (size_t)27 * cin * cout));
    CHK(sc.get(&status, 1));
    GBSW_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    CHK(to_blocked(gy, g.NZ, H, W, cout, gyb, cout / 8, 0, s));
    CHK(pack_weights(w, cin, cout, 1, wp, s));
    if (mask) {
        CHK(sc.get(&mb, nv * cin));
        CHK(to_blocked(mask, g.NZ, H, W, cin, mb, cin / 8, 0, s));
    }
    ConvCall c{};
    CHK(conv_tensor_map(gyb, g, cout / 8, &c.xmap));
    g.mask_cg_total = cin / 8;
    c.geom = g;
    c.wpack = wp;
    c.y_f32 = gx;
    c.mask = mb;
    c.epi = mask ? EPI_MASK : EPI_RAW;
    c.status = status;
    CHK(launch_conv(cout, cin, c, s));
    return finish(status, s);
}

extern "C" gbsw_status unet_conv3d_bwd_weight(int nsamples, int D, int H, int W, int cin, int cout, const float *x,
                                              const float *gy, float *dw, float *db, void *stream)
{
    const int cin_k = cin == 2 ? 16 : cin;  // two input channels run zero-padded to 16, as the first layer does
    if (!x || !gy || !dw || !db || nsamples < 1 || cout > 64 || !pair_ok(cin_k, cout) || (cin_k == 16 && cout == 64))
        return GBSW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ConvGeom g;
    CHK(conv_geometry(nsamples * D, D, H, W, &g));
    const size_t nv = (size_t)nsamples * D * H * W;
    Scratch sc;
    bf16 *xb = nullptr, *gyb = nullptr;
    int *status = nullptr;
    CHK(sc.get(&xb, nv * cin_k));
    CHK(sc.get(&gyb, nv * cout));
    CHK(sc.get(&status, 1));
    GBSW_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    GBSW_CUDA_TRY(cudaMemsetAsync(xb, 0, nv * cin_k * sizeof(bf16), s));
    GBSW_CUDA_TRY(cudaMemsetAsync(dw, 0, (size_t)27 * cin * cout * sizeof(float), s));
    GBSW_CUDA_TRY(cudaMemsetAsync(db, 0, (size_t)cout * sizeof(float), s));
    CHK(to_blocked(x, g.NZ, H, W, cin, xb, cin_k / 8, 0, s));
    CHK(to_blocked(gy, g.NZ, H, W, cout, gyb, cout / 8, 0, s));
    WgradCall c{};
    CHK(conv_tensor_map(xb, g, cin_k / 8, &c.xmap));
    CHK(conv_tensor_map(gyb, g, cout / 8, &c.gmap));
    c.geom = g;
    c.dw = dw;
    c.cin_store = cin;
    c.status = status;
    CHK(launch_wgrad_tc(cin_k, cout, c, s));
    CHK(launch_bias_grad(gyb, cout / 8, 0, (long long)nv, H, W, cout, db, s));
    return finish(status, s);
}

extern "C" gbsw_status unet_glue(int op, int nsamples, int D, int H, int W, int C, const float *a, const float *b,
                                 const float *c, float *out, void *stream)
{
    if (op < 0 || op > 3 || nsamples < 1 || D < 1 || H < 1 || W < 1 || C < 8 || C > 64 || C % 8 || !a || !out)
        return GBSW_ERR_ARG;
    if ((op == 0 || op == 3) && (D % 2 || H % 2 || W % 2)) return GBSW_ERR_ARG;
    if (op == 3 && (!b || !c)) return GBSW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int NZ = nsamples * D;
    const size_t nv = (size_t)NZ * H * W;       // voxels of the (D, H, W) grid
    const size_t nc = nv / 8, nf = nv * 8;      // of the grid halved / doubled
    const int cg = C / 8;
    Scratch sc;
    bf16 *ab = nullptr, *bb = nullptr, *cb = nullptr, *ob = nullptr;
    if (op == 0) {  // pool: a (D, H, W) -> out (D/2, H/2, W/2)
        CHK(sc.get(&ab, nv * C));
        CHK(sc.get(&ob, nc * C));
        CHK(to_blocked(a, NZ, H, W, C, ab, cg, 0, s));
        CHK(launch_pool(ab, cg, 0, NZ, H, W, C, ob, cg, 0, s));
        CHK(from_blocked(ob, NZ / 2, H / 2, W / 2, C, cg, 0, out, s));
    } else if (op == 1) {  // upsample: a (D, H, W) -> out (2D, 2H, 2W)
        CHK(sc.get(&ab, nv * C));
        CHK(sc.get(&ob, nf * C));
        CHK(to_blocked(a, NZ, H, W, C, ab, cg, 0, s));
        CHK(launch_upsample(ab, cg, 0, NZ, H, W, C, ob, cg, 0, s));
        CHK(from_blocked(ob, 2 * NZ, 2 * H, 2 * W, C, cg, 0, out, s));
    } else if (op == 2) {  // upsample adjoint: a (2D, 2H, 2W) -> out (D, H, W)
        CHK(sc.get(&ab, nf * C));
        CHK(sc.get(&ob, nv * C));
        CHK(to_blocked(a, 2 * NZ, 2 * H, 2 * W, C, ab, cg, 0, s));
        CHK(launch_upsample_bwd(ab, cg, 0, NZ, H, W, C, ob, cg, 0, s));
        CHK(from_blocked(ob, NZ, H, W, C, cg, 0, out, s));
    } else {  // (a + pool adjoint of b) * [c > 0]: a, c, out (D, H, W), b (D/2, H/2, W/2)
        CHK(sc.get(&ab, nv * C));
        CHK(sc.get(&bb, nc * C));
        CHK(sc.get(&cb, nv * C));
        CHK(sc.get(&ob, nv * C));
        CHK(to_blocked(a, NZ, H, W, C, ab, cg, 0, s));
        CHK(to_blocked(b, NZ / 2, H / 2, W / 2, C, bb, cg, 0, s));
        CHK(to_blocked(c, NZ, H, W, C, cb, cg, 0, s));
        CHK(launch_pool_bwd_add_mask(ab, cg, 0, bb, cg, 0, cb, cg, 0, NZ, H, W, C, ob, cg, 0, s));
        CHK(from_blocked(ob, NZ, H, W, C, cg, 0, out, s));
    }
    GBSW_CUDA_TRY(cudaStreamSynchronize(s));
    return GBSW_OK;
}

extern "C" gbsw_status unet_head(long long nvox, const float *d1, const float *hw, const float *hb,
                                 const float *target, float *out, float *g_hw, float *g_hb, float *g_d1, double *loss,
                                 void *stream)
{
    if (nvox < 1 || nvox > (1LL << 30) || !d1 || !hw || !hb || !out) return GBSW_ERR_ARG;
    if (target && (!g_hw || !g_hb || !g_d1 || !loss)) return GBSW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int W = (int)nvox;  // one plane of one row: voxel v at x = v
    Scratch sc;
    bf16 *db = nullptr, *gb = nullptr;
    CHK(sc.get(&db, (size_t)nvox * 16));
    CHK(to_blocked(d1, 1, 1, W, 16, db, 2, 0, s));
    CHK(launch_head_fwd(db, 2, 0, nvox, 1, W, hw, hb, out, s));
    if (target) {
        CHK(sc.get(&gb, (size_t)nvox * 16));
        GBSW_CUDA_TRY(cudaMemsetAsync(g_hw, 0, 16 * sizeof(float), s));
        GBSW_CUDA_TRY(cudaMemsetAsync(g_hb, 0, sizeof(float), s));
        GBSW_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(double), s));
        CHK(launch_head_bwd(db, 2, 0, nvox, 1, W, out, target, hw, g_hw, g_hb, gb, loss, s));
        CHK(from_blocked(gb, 1, 1, W, 16, 2, 0, g_d1, s));
    }
    GBSW_CUDA_TRY(cudaStreamSynchronize(s));
    return GBSW_OK;
}

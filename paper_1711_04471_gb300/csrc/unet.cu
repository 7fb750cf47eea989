// The warm-start U-Net: parameters, activations, forward / backward
// schedules, Adam training and the LES hook (see include/gbsw.h).
//
//   l1a 2->16 (input zero-padded to 16), l1b 16->16    -> s1   full resolution
//   pool, l2a 16->32, l2b 32->32                        -> s2   1/2
//   pool, l3a 32->64, l3b 64->32                                1/4
//   upsample, cat [up, s2] (64), l2c 64->16                     1/2
//   upsample, cat [up, s1] (32), l1c 32->16                     full
//   head 1x1x1 16->1
// Every 3x3x3 layer runs on the tcgen05 kernels: forward, backward-data
// with flipped weights and weight gradients (l1a's two input channels are
// zero-padded to 16 in a BF16 copy of the input).  Concatenations are
// free: the producers write into channel-group ranges of one buffer
// (u1 = [up(d2), s1], u2 = [up(b3), s2]).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "unet_ops.cuh"
#include "warmstart.cuh"

using namespace gbsw;

namespace {

struct LayerDef {
    int cin, cout;
};
constexpr int NLAYERS = 8;
constexpr LayerDef LAYERS[NLAYERS] = {{2, 16}, {16, 16}, {16, 32}, {32, 32}, {32, 64}, {64, 32}, {64, 16}, {32, 16}};
enum { L1A = 0, L1B, L2A, L2B, L3A, L3B, L2C, L1C };

int param_count()
{
    int n = 0;
    for (const auto &l : LAYERS) n += 27 * l.cin * l.cout + l.cout;
    return n + 16 + 1;
}

struct Acts {
    int N, D, H, W;
    ConvGeom g[3];             // levels 1..3
    long long nvox;            // full-resolution voxels
    float *xin = nullptr, *out = nullptr;
    bf16 *x16 = nullptr;       // xin as C8-blocked BF16, channels 2..15 zero (l1a's padded input)
    double *ws = nullptr;      // warm start: block means r_c, p_c (nvox each) and the scale
    bf16 *a1a, *u1, *p1, *a2a, *u2, *p2, *a3a, *b3, *d2, *d1;
    bf16 *g_d1 = nullptr, *g_u1, *g_d2, *g_u2, *g_b3, *g_a3a, *g_p2, *g_s2, *g_a2a, *g_p1, *g_s1, *g_a1a;
    CUtensorMap m_fwd[NLAYERS];  // input map of each layer's forward conv (and of its weight gradient)
    CUtensorMap m_bwd[NLAYERS];  // map of each layer's gz: input of its backward-data conv and of its weight gradient
    std::vector<void *> allocs;
    bool train = false;
};

}  // namespace

struct gbsw_unet {
    int nparams;
    int w_off[NLAYERS], b_off[NLAYERS], hw_off, hb_off;
    float *params, *grads, *m, *v;
    bf16 *pack_fwd[NLAYERS], *pack_bwd[NLAYERS];
    bool packs_dirty;
    int adam_step;
    int *status;
    double *loss;
    cudaStream_t stream;
    std::map<std::tuple<int, int, int, int>, Acts *> acts;
};

namespace {

void free_acts(Acts *a)
{
    for (void *p : a->allocs) cudaFree(p);
    delete a;
}

template <typename T>
gbsw_status alloc(Acts *a, T **p, size_t n)
{
    GBSW_CUDA_TRY(cudaMalloc((void **)p, n * sizeof(T)));
    a->allocs.push_back(*p);
    return GBSW_OK;
}

gbsw_status make_acts(int N, int D, int H, int W, bool train, Acts **out)
{
    if (N < 1 || D % 4 || H % 4 || W % 4) return GBSW_ERR_ARG;
    Acts *a = new (std::nothrow) Acts();
    if (!a) return GBSW_ERR_OOM;
    a->N = N;
    a->D = D;
    a->H = H;
    a->W = W;
    gbsw_status st = GBSW_OK;
    for (int l = 0; l < 3 && st == GBSW_OK; ++l) {
        const int s = 1 << l;
        st = conv_geometry(N * (D / s), D / s, H / s, W / s, &a->g[l]);
    }
    if (st != GBSW_OK) {
        delete a;
        return st;
    }
    const long long v1 = (long long)N * D * H * W, v2 = v1 / 8, v3 = v2 / 8;
    a->nvox = v1;
    auto B = [&](bf16 **p, long long vox, int C) {
        if (st == GBSW_OK) st = alloc(a, p, (size_t)vox * C);
    };
    if (st == GBSW_OK) st = alloc(a, &a->xin, (size_t)v1 * 2);
    if (st == GBSW_OK) st = alloc(a, &a->out, (size_t)v1);
    if (st == GBSW_OK && N == 1) st = alloc(a, &a->ws, (size_t)(2 * v1 + 1));
    B(&a->x16, v1, 16);
    // the padding channels stay zero for the life of the buffer; finish
    // the fill before any stream (the caller's or the LES's) uses it
    if (st == GBSW_OK && (cudaMemset(a->x16, 0, (size_t)v1 * 16 * sizeof(bf16)) != cudaSuccess ||
                          cudaDeviceSynchronize() != cudaSuccess))
        st = GBSW_ERR_CUDA;
    B(&a->a1a, v1, 16);
    B(&a->u1, v1, 32);
    B(&a->p1, v2, 16);
    B(&a->a2a, v2, 32);
    B(&a->u2, v2, 64);
    B(&a->p2, v3, 32);
    B(&a->a3a, v3, 64);
    B(&a->b3, v3, 32);
    B(&a->d2, v2, 16);
    B(&a->d1, v1, 16);
    if (train) {
        B(&a->g_d1, v1, 16);
        B(&a->g_u1, v1, 32);
        B(&a->g_d2, v2, 16);
        B(&a->g_u2, v2, 64);
        B(&a->g_b3, v3, 32);
        B(&a->g_a3a, v3, 64);
        B(&a->g_p2, v3, 32);
        B(&a->g_s2, v2, 32);
        B(&a->g_a2a, v2, 32);
        B(&a->g_p1, v2, 16);
        B(&a->g_s1, v1, 16);
        B(&a->g_a1a, v1, 16);
    }
    a->train = train;
    const ConvGeom &g1 = a->g[0], &g2 = a->g[1], &g3 = a->g[2];
    // forward inputs
    struct M {
        int layer;
        const bf16 *p;
        const ConvGeom *g;
        int cg;
    };
    const M fwd[] = {{L1A, a->x16, &g1, 2}, {L1B, a->a1a, &g1, 2}, {L2A, a->p1, &g2, 2}, {L2B, a->a2a, &g2, 4},
                     {L3A, a->p2, &g3, 4},  {L3B, a->a3a, &g3, 8}, {L2C, a->u2, &g2, 8}, {L1C, a->u1, &g1, 4}};
    for (const M &m : fwd)
        if (st == GBSW_OK) st = conv_tensor_map(m.p, *m.g, m.cg, &a->m_fwd[m.layer]);
    if (train) {
        // the gz of each layer (Cout channels): backward-data and weight-gradient input
        const M bwd[] = {{L1A, a->g_a1a, &g1, 2}, {L1B, a->g_s1, &g1, 2}, {L2A, a->g_a2a, &g2, 4},
                         {L2B, a->g_s2, &g2, 4},  {L3A, a->g_a3a, &g3, 8}, {L3B, a->g_b3, &g3, 4},
                         {L2C, a->g_d2, &g2, 2},  {L1C, a->g_d1, &g1, 2}};
        for (const M &m : bwd)
            if (st == GBSW_OK) st = conv_tensor_map(m.p, *m.g, m.cg, &a->m_bwd[m.layer]);
    }
    if (st != GBSW_OK) {
        free_acts(a);
        return st;
    }
    *out = a;
    return GBSW_OK;
}

gbsw_status get_acts(gbsw_unet *u, int N, int D, int H, int W, bool train, Acts **out)
{
    auto key = std::make_tuple(N, D, H, W);
    auto it = u->acts.find(key);
    if (it != u->acts.end() && (it->second->train || !train)) {
        *out = it->second;
        return GBSW_OK;
    }
    if (it != u->acts.end()) {
        cudaStreamSynchronize(u->stream);
        free_acts(it->second);
        u->acts.erase(it);
    }
    Acts *a = nullptr;
    gbsw_status st = make_acts(N, D, H, W, train, &a);
    if (st != GBSW_OK) return st;
    u->acts[key] = a;
    *out = a;
    return GBSW_OK;
}

#define TRY(x)                          \
    do {                                \
        gbsw_status _s = (x);           \
        if (_s != GBSW_OK) return _s;   \
    } while (0)

gbsw_status repack(gbsw_unet *u, cudaStream_t s)
{
    if (!u->packs_dirty) return GBSW_OK;
    TRY(pack_weights_padded(u->params + u->w_off[L1A], LAYERS[L1A].cin, 16, LAYERS[L1A].cout, 0, u->pack_fwd[L1A], s));
    for (int l = 1; l < NLAYERS; ++l) {
        gbsw_status st = pack_weights(u->params + u->w_off[l], LAYERS[l].cin, LAYERS[l].cout, 0, u->pack_fwd[l], s);
        if (st == GBSW_OK)
            st = pack_weights(u->params + u->w_off[l], LAYERS[l].cin, LAYERS[l].cout, 1, u->pack_bwd[l], s);
        if (st != GBSW_OK) return st;
    }
    u->packs_dirty = false;
    return GBSW_OK;
}

// One tcgen05 conv: input map, level geometry, output buffer and channel
// range, epilogue (bias for EPI_BIAS_RELU, mask tensor for EPI_MASK).
gbsw_status conv(gbsw_unet *u, int cin, int cout, const CUtensorMap &map, const bf16 *wpack, const float *bias,
                 const ConvGeom &g, bf16 *y, int y_cg_total, int y_cg0, int epi, const bf16 *mask, int m_cg_total,
                 int m_cg0, cudaStream_t s)
{
    ConvCall c{};
    c.xmap = map;
    c.wpack = wpack;
    c.bias = bias;
    c.y = y;
    c.y_f32 = nullptr;
    c.mask = mask;
    c.geom = g;
    c.geom.out_cg_total = y_cg_total;
    c.geom.out_cg0 = y_cg0;
    c.geom.mask_cg_total = m_cg_total;
    c.geom.mask_cg0 = m_cg0;
    c.epi = epi;
    c.status = u->status;
    return launch_conv(cin, cout, c, s);
}


// Forward pass on a->xin; writes a->out.
gbsw_status forward(gbsw_unet *u, Acts *a, cudaStream_t s)
{
    TRY(repack(u, s));
    const ConvGeom &g1 = a->g[0], &g2 = a->g[1], &g3 = a->g[2];
    float *P = u->params;
    auto W = [&](int l) { return u->pack_fwd[l]; };
    auto Bv = [&](int l) { return P + u->b_off[l]; };
    TRY(to_blocked(a->xin, g1.NZ, g1.H, g1.W, 2, a->x16, 2, 0, s));
    TRY(conv(u, 16, 16, a->m_fwd[L1A], W(L1A), Bv(L1A), g1, a->a1a, 2, 0, EPI_BIAS_RELU, nullptr, 0, 0, s));
    TRY(conv(u, 16, 16, a->m_fwd[L1B], W(L1B), Bv(L1B), g1, a->u1, 4, 2, EPI_BIAS_RELU, nullptr, 0, 0, s));
    TRY(launch_pool(a->u1, 4, 2, g1.NZ, g1.H, g1.W, 16, a->p1, 2, 0, s));
    TRY(conv(u, 16, 32, a->m_fwd[L2A], W(L2A), Bv(L2A), g2, a->a2a, 4, 0, EPI_BIAS_RELU, nullptr, 0, 0, s));
    TRY(conv(u, 32, 32, a->m_fwd[L2B], W(L2B), Bv(L2B), g2, a->u2, 8, 4, EPI_BIAS_RELU, nullptr, 0, 0, s));
    TRY(launch_pool(a->u2, 8, 4, g2.NZ, g2.H, g2.W, 32, a->p2, 4, 0, s));
    TRY(conv(u, 32, 64, a->m_fwd[L3A], W(L3A), Bv(L3A), g3, a->a3a, 8, 0, EPI_BIAS_RELU, nullptr, 0, 0, s));
    TRY(conv(u, 64, 32, a->m_fwd[L3B], W(L3B), Bv(L3B), g3, a->b3, 4, 0, EPI_BIAS_RELU, nullptr, 0, 0, s));
    TRY(launch_upsample(a->b3, 4, 0, g3.NZ, g3.H, g3.W, 32, a->u2, 8, 0, s));
    TRY(conv(u, 64, 16, a->m_fwd[L2C], W(L2C), Bv(L2C), g2, a->d2, 2, 0, EPI_BIAS_RELU, nullptr, 0, 0, s));
    TRY(launch_upsample(a->d2, 2, 0, g2.NZ, g2.H, g2.W, 16, a->u1, 4, 0, s));
    TRY(conv(u, 32, 16, a->m_fwd[L1C], W(L1C), Bv(L1C), g1, a->d1, 2, 0, EPI_BIAS_RELU, nullptr, 0, 0, s));
    TRY(launch_head_fwd(a->d1, 2, 0, a->nvox, g1.H, g1.W, P + u->hw_off, P + u->hb_off, a->out, s));
    return GBSW_OK;
}

// Weight and bias gradients of layer l from its input (m_fwd[l]) and its
// gz (m_bwd[l], the C8-blocked tensor gz with cout / 8 channel groups).
gbsw_status wgrad(gbsw_unet *u, Acts *a, int l, const ConvGeom &g, const bf16 *gz, cudaStream_t s)
{
    WgradCall c{};
    c.xmap = a->m_fwd[l];
    c.gmap = a->m_bwd[l];
    c.geom = g;
    c.dw = u->grads + u->w_off[l];
    c.cin_store = LAYERS[l].cin;
    c.status = u->status;
    const int cin = l == L1A ? 16 : LAYERS[l].cin;
    TRY(launch_wgrad_tc(cin, LAYERS[l].cout, c, s));
    const long long nvox = (long long)g.NZ * g.H * g.W;
    return launch_bias_grad(gz, LAYERS[l].cout / 8, 0, nvox, g.H, g.W, LAYERS[l].cout, u->grads + u->b_off[l], s);
}

// Backward pass of MSE(out, target) after forward(); accumulates into
// u->grads (zeroed here) and adds the loss to *u->loss.
gbsw_status backward(gbsw_unet *u, Acts *a, const float *target, cudaStream_t s)
{
    const ConvGeom &g1 = a->g[0], &g2 = a->g[1], &g3 = a->g[2];
    float *G = u->grads;
    auto WB = [&](int l) { return u->pack_bwd[l]; };
    GBSW_CUDA_TRY(cudaMemsetAsync(G, 0, (size_t)u->nparams * sizeof(float), s));
    TRY(launch_head_bwd(a->d1, 2, 0, a->nvox, g1.H, g1.W, a->out, target, u->params + u->hw_off, G + u->hw_off,
                        G + u->hb_off, a->g_d1, u->loss, s));
    // l1c: input u1 = [up(d2), s1]
    TRY(wgrad(u, a, L1C, g1, a->g_d1, s));
    TRY(conv(u, 16, 32, a->m_bwd[L1C], WB(L1C), nullptr, g1, a->g_u1, 4, 0, EPI_MASK, a->u1, 4, 0, s));
    TRY(launch_upsample_bwd(a->g_u1, 4, 0, g2.NZ, g2.H, g2.W, 16, a->g_d2, 2, 0, s));
    // l2c: input u2 = [up(b3), s2]
    TRY(wgrad(u, a, L2C, g2, a->g_d2, s));
    TRY(conv(u, 16, 64, a->m_bwd[L2C], WB(L2C), nullptr, g2, a->g_u2, 8, 0, EPI_MASK, a->u2, 8, 0, s));
    TRY(launch_upsample_bwd(a->g_u2, 8, 0, g3.NZ, g3.H, g3.W, 32, a->g_b3, 4, 0, s));
    // l3b, l3a
    TRY(wgrad(u, a, L3B, g3, a->g_b3, s));
    TRY(conv(u, 32, 64, a->m_bwd[L3B], WB(L3B), nullptr, g3, a->g_a3a, 8, 0, EPI_MASK, a->a3a, 8, 0, s));
    TRY(wgrad(u, a, L3A, g3, a->g_a3a, s));
    TRY(conv(u, 64, 32, a->m_bwd[L3A], WB(L3A), nullptr, g3, a->g_p2, 4, 0, EPI_RAW, nullptr, 0, 0, s));
    // s2 receives the concat gradient and the pooled path
    TRY(launch_pool_bwd_add_mask(a->g_u2, 8, 4, a->g_p2, 4, 0, a->u2, 8, 4, g2.NZ, g2.H, g2.W, 32, a->g_s2, 4, 0, s));
    TRY(wgrad(u, a, L2B, g2, a->g_s2, s));
    TRY(conv(u, 32, 32, a->m_bwd[L2B], WB(L2B), nullptr, g2, a->g_a2a, 4, 0, EPI_MASK, a->a2a, 4, 0, s));
    TRY(wgrad(u, a, L2A, g2, a->g_a2a, s));
    TRY(conv(u, 32, 16, a->m_bwd[L2A], WB(L2A), nullptr, g2, a->g_p1, 2, 0, EPI_RAW, nullptr, 0, 0, s));
    TRY(launch_pool_bwd_add_mask(a->g_u1, 4, 2, a->g_p1, 2, 0, a->u1, 4, 2, g1.NZ, g1.H, g1.W, 16, a->g_s1, 2, 0, s));
    TRY(wgrad(u, a, L1B, g1, a->g_s1, s));
    TRY(conv(u, 16, 16, a->m_bwd[L1B], WB(L1B), nullptr, g1, a->g_a1a, 2, 0, EPI_MASK, a->a1a, 2, 0, s));
    TRY(wgrad(u, a, L1A, g1, a->g_a1a, s));
    return GBSW_OK;
}

// He-normal initial weights from SplitMix64 + Box-Muller (host).
struct HostRng {
    unsigned long long s;
    unsigned long long next()
    {
        unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal() { return sqrt(-2.0 * log(uniform())) * cos(6.283185307179586 * uniform()); }
};

}  // namespace

// Hook used by the LES step (declared in unet_ops.cuh's companion below).
namespace gbsw {
bool unet_shape_ok(int D, int H, int W)
{
    if (D < 4 || H < 4 || W < 4 || D % 4 || H % 4 || W % 4) return false;
    ConvGeom g;
    for (int l = 0; l < 3; ++l) {
        const int s = 1 << l;
        if (conv_geometry(D / s, D / s, H / s, W / s, &g) != GBSW_OK) return false;
    }
    return true;
}

gbsw_status unet_warm_start(gbsw_unet *u, const float *b, double *p, const PadDims &pd, double dx, int f,
                            double *scratch, cudaStream_t s)
{
    if (!ws_factor_ok(pd.nx, pd.ny, pd.nz, f)) return GBSW_ERR_ARG;
    Acts *a = nullptr;
    TRY(get_acts(u, 1, pd.nz / f, pd.ny / f, pd.nx / f, false, &a));
    const WsGrid g{pd.nx, pd.ny, pd.nz, pd.pitch, pd.plane, pd.plane + pd.pitch + 1, pd.plane * (pd.nz + 2)};
    const long long nc = a->nvox;
    TRY(launch_ws_restrict(b, p, g, dx, f, scratch, a->ws, a->ws + nc, s));
    TRY(launch_ws_prepare(a->ws, a->ws + nc, nc, (f * dx) * (f * dx), a->xin, a->ws + 2 * nc, s));
    TRY(forward(u, a, s));
    TRY(launch_ws_prolong(a->out, g, f, a->ws + 2 * nc, p, s));
    return GBSW_OK;
}
}  // namespace gbsw

extern "C" {

int unet_num_params(void) { return param_count(); }

gbsw_status unet_create(unsigned long long seed, void *stream, gbsw_unet **out)
{
    if (!out) return GBSW_ERR_ARG;
    if (fault_injected("alloc")) return GBSW_ERR_OOM;
    gbsw_unet *u = new (std::nothrow) gbsw_unet();
    if (!u) return GBSW_ERR_OOM;
    u->stream = (cudaStream_t)stream;
    int off = 0;
    for (int l = 0; l < NLAYERS; ++l) {
        u->w_off[l] = off;
        off += 27 * LAYERS[l].cin * LAYERS[l].cout;
        u->b_off[l] = off;
        off += LAYERS[l].cout;
    }
    u->hw_off = off;
    u->hb_off = off + 16;
    u->nparams = off + 17;
    std::vector<float> h(u->nparams, 0.0f);
    HostRng rng{seed};
    for (int l = 0; l < NLAYERS; ++l) {
        const double sd = sqrt(2.0 / (27.0 * LAYERS[l].cin));
        for (int q = 0; q < 27 * LAYERS[l].cin * LAYERS[l].cout; ++q) h[u->w_off[l] + q] = (float)(sd * rng.normal());
    }
    for (int c = 0; c < 16; ++c) h[u->hw_off + c] = (float)(0.25 * rng.normal());
    auto fail = [&](gbsw_status st) {
        unet_destroy(u);
        return st;
    };
    const size_t pb = (size_t)u->nparams * sizeof(float);
    if (cudaMalloc((void **)&u->params, pb) != cudaSuccess || cudaMalloc((void **)&u->grads, pb) != cudaSuccess ||
        cudaMalloc((void **)&u->m, pb) != cudaSuccess || cudaMalloc((void **)&u->v, pb) != cudaSuccess ||
        cudaMalloc((void **)&u->status, sizeof(int)) != cudaSuccess ||
        cudaMalloc((void **)&u->loss, sizeof(double)) != cudaSuccess)
        return fail(GBSW_ERR_OOM);
    if (cudaMalloc((void **)&u->pack_fwd[L1A], (size_t)27 * 16 * 16 * sizeof(bf16)) != cudaSuccess)
        return fail(GBSW_ERR_OOM);  // l1a: input channels padded to 16; no backward-data pack
    for (int l = 1; l < NLAYERS; ++l) {
        const size_t n = (size_t)27 * LAYERS[l].cin * LAYERS[l].cout * sizeof(bf16);
        if (cudaMalloc((void **)&u->pack_fwd[l], n) != cudaSuccess || cudaMalloc((void **)&u->pack_bwd[l], n) != cudaSuccess)
            return fail(GBSW_ERR_OOM);
    }
    cudaError_t e = cudaMemcpyAsync(u->params, h.data(), pb, cudaMemcpyHostToDevice, u->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->m, 0, pb, u->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->v, 0, pb, u->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->grads, 0, pb, u->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->status, 0, sizeof(int), u->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
    if (e != cudaSuccess) {
        record_cuda_error(e, "unet_create", __FILE__, __LINE__);
        return fail(GBSW_ERR_CUDA);
    }
    u->packs_dirty = true;
    *out = u;
    return GBSW_OK;
}

gbsw_status unet_get_params(gbsw_unet *u, float *host, int n)
{
    if (!u || !host || n != u->nparams) return GBSW_ERR_ARG;
    GBSW_CUDA_TRY(cudaMemcpyAsync(host, u->params, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, u->stream));
    GBSW_CUDA_TRY(cudaStreamSynchronize(u->stream));
    return GBSW_OK;
}

gbsw_status unet_set_params(gbsw_unet *u, const float *host, int n)
{
    if (!u || !host || n != u->nparams) return GBSW_ERR_ARG;
    GBSW_CUDA_TRY(cudaMemcpyAsync(u->params, host, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, u->stream));
    GBSW_CUDA_TRY(cudaStreamSynchronize(u->stream));
    u->packs_dirty = true;
    return GBSW_OK;
}

static gbsw_status check_status(gbsw_unet *u)
{
    int h = 0;
    GBSW_CUDA_TRY(cudaMemcpyAsync(&h, u->status, sizeof(int), cudaMemcpyDeviceToHost, u->stream));
    GBSW_CUDA_TRY(cudaStreamSynchronize(u->stream));
    return dev_status_to_gbsw(h);
}

gbsw_status unet_forward(gbsw_unet *u, int n, int D, int H, int W, const float *x, float *y)
{
    gbsw::NvtxRange nvtx_range("unet_forward");
    if (!u || !x || !y) return GBSW_ERR_ARG;
    Acts *a = nullptr;
    TRY(get_acts(u, n, D, H, W, false, &a));
    GBSW_CUDA_TRY(cudaMemcpyAsync(a->xin, x, (size_t)a->nvox * 2 * sizeof(float), cudaMemcpyDeviceToDevice, u->stream));
    TRY(forward(u, a, u->stream));
    GBSW_CUDA_TRY(cudaMemcpyAsync(y, a->out, (size_t)a->nvox * sizeof(float), cudaMemcpyDeviceToDevice, u->stream));
    return check_status(u);
}

gbsw_status unet_infer(gbsw_unet *u, int n, int D, int H, int W, const float *x, float *y)
{
    return unet_forward(u, n, D, H, W, x, y);
}

// Loss and gradients (no update); grads_host may be NULL.
gbsw_status unet_gradients(gbsw_unet *u, int n, int D, int H, int W, const float *x, const float *target,
                           float *grads_host, double *loss)
{
    gbsw::NvtxRange nvtx_range("unet_gradients");
    if (!u || !x || !target) return GBSW_ERR_ARG;
    Acts *a = nullptr;
    TRY(get_acts(u, n, D, H, W, true, &a));
    GBSW_CUDA_TRY(cudaMemcpyAsync(a->xin, x, (size_t)a->nvox * 2 * sizeof(float), cudaMemcpyDeviceToDevice, u->stream));
    GBSW_CUDA_TRY(cudaMemsetAsync(u->loss, 0, sizeof(double), u->stream));
    TRY(forward(u, a, u->stream));
    TRY(backward(u, a, target, u->stream));
    if (grads_host)
        GBSW_CUDA_TRY(cudaMemcpyAsync(grads_host, u->grads, (size_t)u->nparams * sizeof(float), cudaMemcpyDeviceToHost,
                                      u->stream));
    double l = 0.0;
    GBSW_CUDA_TRY(cudaMemcpyAsync(&l, u->loss, sizeof(double), cudaMemcpyDeviceToHost, u->stream));
    gbsw_status st = check_status(u);
    if (loss) *loss = l;
    return st;
}

gbsw_status unet_train_step(gbsw_unet *u, int n, int D, int H, int W, const float *x, const float *target, float lr,
                            double *loss)
{
    gbsw::NvtxRange nvtx_range("unet_train_step");
    if (!u || !x || !target || !(lr > 0)) return GBSW_ERR_ARG;
    Acts *a = nullptr;
    TRY(get_acts(u, n, D, H, W, true, &a));
    GBSW_CUDA_TRY(cudaMemcpyAsync(a->xin, x, (size_t)a->nvox * 2 * sizeof(float), cudaMemcpyDeviceToDevice, u->stream));
    GBSW_CUDA_TRY(cudaMemsetAsync(u->loss, 0, sizeof(double), u->stream));
    TRY(forward(u, a, u->stream));
    TRY(backward(u, a, target, u->stream));
    u->adam_step += 1;
    TRY(launch_adam(u->params, u->grads, u->m, u->v, u->nparams, lr, u->adam_step, u->stream));
    u->packs_dirty = true;
    if (loss) {
        GBSW_CUDA_TRY(cudaMemcpyAsync(loss, u->loss, sizeof(double), cudaMemcpyDeviceToHost, u->stream));
        return check_status(u);
    }
    return GBSW_OK;
}

void unet_destroy(gbsw_unet *u)
{
    if (!u) return;
    cudaStreamSynchronize(u->stream);
    for (auto &kv : u->acts) free_acts(kv.second);
    for (int l = 0; l < NLAYERS; ++l) {
        cudaFree(u->pack_fwd[l]);
        cudaFree(u->pack_bwd[l]);
    }
    cudaFree(u->params);
    cudaFree(u->grads);
    cudaFree(u->m);
    cudaFree(u->v);
    cudaFree(u->status);
    cudaFree(u->loss);
    delete u;
}

}  // extern "C"

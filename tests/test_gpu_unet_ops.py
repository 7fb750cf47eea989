"""Every kernel of the warm-start U-Net on its own, through the C ABI,
against the FP64 oracle (oracle/unet.py).

Operands are BF16-representable, so each tensor-core product is exact in
FP32 and the convolutions, their backward-data pass and the weight
gradients differ from the oracle only by the FP32 summation order: relative
L2 error <= 1e-5.  The glue kernels (pooling, upsampling and their
adjoints) store BF16: on dyadic inputs whose sums are exact in FP32 they
must equal the BF16-rounded oracle bit for bit.  The head computes in FP32
(<= 1e-5); its BF16 input gradient may differ from the rounded oracle by
one BF16 unit where dL/dout, formed in FP32, lies at a rounding boundary.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from oracle import unet as OU

from unet_bf16 import bf16

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def L():
    import paper_1711_04471_gb300 as P
    P.build()
    from paper_1711_04471_gb300 import _native as N
    oracle.lib()
    return N


_keep = []


def dev(a):
    """A CUDA copy of a, kept alive until the next test (the C calls below
    receive only its address, so a temporary must not be freed and reused
    before the kernel has read it)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    _keep.append(t)
    return t


@pytest.fixture(autouse=True)
def _release():
    yield
    _keep.clear()


def ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300)


# layer pairs of the network and tile geometries: whole 128-voxel rows, tiles of several rows, tiles of
# several planes (coarse levels), partial last tiles and tiles crossing from one sample into the next
LAYER_PAIRS = [(16, 16), (16, 32), (32, 32), (32, 64), (64, 32), (64, 16), (32, 16)]
GEOMS = [(2, 3, 4, 32), (1, 4, 8, 16), (3, 2, 4, 4), (1, 2, 2, 128), (2, 4, 8, 8)]


def _cases():
    out = []
    for k, (ci, co) in enumerate(LAYER_PAIRS):
        for g in (GEOMS[k % len(GEOMS)], GEOMS[(k + 2) % len(GEOMS)]):
            out.append((g, ci, co))
    return out


@pytest.mark.parametrize("shape,cin,cout", _cases())
def test_conv_backward_data(L, shape, cin, cout):
    import torch
    n, D, H, W = shape
    rng = np.random.default_rng(cin * 7 + cout + D)
    gy = bf16(rng.standard_normal((n, D, H, W, cout)))
    w = bf16(rng.standard_normal((27, cout, cin)) * 0.2)
    mask = rng.standard_normal((n, D, H, W, cin))
    for use_mask in (False, True):
        gx = torch.empty((n, D, H, W, cin), device="cuda")
        L.check(L.lib().unet_conv3d_bwd_data(n, D, H, W, cin, cout, ptr(dev(gy)), ptr(dev(w)),
                                             ptr(dev(mask)) if use_mask else None, ptr(gx), None),
                "unet_conv3d_bwd_data")
        ref = np.stack([OU.conv3d_bwd_data(gy[k], w, cin) for k in range(n)])
        if use_mask:
            ref = ref * (bf16(mask) > 0)
        got = gx.cpu().numpy()
        assert rel(got, ref) <= TOL, (use_mask, rel(got, ref))
        if use_mask:
            assert np.all(got[bf16(mask) <= 0] == 0)


@pytest.mark.parametrize("shape,cin,cout", _cases() + [((2, 4, 8, 16), 2, 16), ((1, 2, 4, 32), 2, 16)])
def test_conv_weight_gradients(L, shape, cin, cout):
    import torch
    n, D, H, W = shape
    rng = np.random.default_rng(cin * 11 + cout + H)
    x = bf16(rng.standard_normal((n, D, H, W, cin)))
    gy = bf16(rng.standard_normal((n, D, H, W, cout)))
    dw = torch.empty((27, cout, cin), device="cuda")
    db = torch.empty(cout, device="cuda")
    L.check(L.lib().unet_conv3d_bwd_weight(n, D, H, W, cin, cout, ptr(dev(x)), ptr(dev(gy)), ptr(dw), ptr(db), None),
            "unet_conv3d_bwd_weight")
    rw, rb = 0.0, 0.0
    for k in range(n):
        a, b = OU.conv3d_bwd_weight(x[k], gy[k])
        rw, rb = rw + a, rb + b
    assert rel(dw.cpu().numpy(), rw) <= TOL, rel(dw.cpu().numpy(), rw)
    assert rel(db.cpu().numpy(), rb) <= TOL


def test_weight_gradients_see_zero_padding_and_sample_edges(L):
    """A weight gradient tap that leaves the grid or the sample reads zeros:
    with x = 1 everywhere and gy = 1 on one voxel at a corner of sample 1,
    dw[tap] counts exactly the taps that land inside that sample."""
    import torch
    n, D, H, W, cin, cout = 2, 4, 8, 16, 16, 16
    x = np.ones((n, D, H, W, cin))
    gy = np.zeros((n, D, H, W, cout))
    gy[1, 0, 0, 0, :] = 1.0
    dw = torch.empty((27, cout, cin), device="cuda")
    db = torch.empty(cout, device="cuda")
    L.check(L.lib().unet_conv3d_bwd_weight(n, D, H, W, cin, cout, ptr(dev(x)), ptr(dev(gy)), ptr(dw), ptr(db), None),
            "unet_conv3d_bwd_weight")
    got = dw.cpu().numpy()
    for tap in range(27):
        dz, dy, dx = tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1
        inside = dz >= 0 and dy >= 0 and dx >= 0
        assert np.all(got[tap] == (1.0 if inside else 0.0)), tap
    assert np.all(db.cpu().numpy() == 1.0)


@pytest.mark.parametrize("shape", [(2, 4, 8, 16), (1, 2, 4, 32), (3, 2, 4, 4)])
def test_first_layer_conv_two_channels(L, shape):
    """l1a: two input channels, run zero-padded to 16 on the tensor cores."""
    import torch
    n, D, H, W = shape
    rng = np.random.default_rng(D * H)
    x = bf16(rng.standard_normal((n, D, H, W, 2)))
    w = bf16(rng.standard_normal((27, 16, 2)) * 0.3)
    b = rng.standard_normal(16).astype(np.float32)
    y = torch.empty((n, D, H, W, 16), device="cuda")
    L.check(L.lib().unet_conv3d(n, D, H, W, 2, 16, ptr(dev(x)), ptr(dev(w)), ptr(dev(b)), 0, None, ptr(y), None),
            "unet_conv3d")
    ref = np.stack([np.maximum(OU.conv3d(x[k], w, b.astype(np.float64)), 0) for k in range(n)])
    assert rel(y.cpu().numpy(), ref) <= TOL


def _dyadic(rng, shape):
    """Values k / 16 with |k| <= 127: exact in BF16, and sums of eight are exact in FP32."""
    return rng.integers(-127, 128, size=shape) / 16.0


@pytest.mark.parametrize("C_", [16, 32, 64])
def test_glue_ops_bitwise(L, C_):
    import torch
    rng = np.random.default_rng(C_)
    n, D, H, W = 2, 4, 8, 6
    a = _dyadic(rng, (n, D, H, W, C_))

    def run(op, shp, a_, b_=None, c_=None, out_shape=None):
        out = torch.empty(out_shape, device="cuda")
        L.check(L.lib().unet_glue(op, n, *shp, C_, ptr(dev(a_)), ptr(None if b_ is None else dev(b_)),
                                  ptr(None if c_ is None else dev(c_)), ptr(out), None), "unet_glue")
        return out.cpu().numpy()

    half = (n, D // 2, H // 2, W // 2, C_)
    dbl = (n, 2 * D, 2 * H, 2 * W, C_)
    got = run(0, (D, H, W), a, out_shape=half)
    assert np.array_equal(got, bf16(np.stack([OU.avgpool2(a[k]) for k in range(n)])))
    got = run(1, (D, H, W), a, out_shape=dbl)
    assert np.array_equal(got, np.stack([OU.upsample2(a[k]) for k in range(n)]))
    a2 = _dyadic(rng, dbl)
    got = run(2, (D, H, W), a2, out_shape=(n, D, H, W, C_))
    assert np.array_equal(got, bf16(np.stack([OU.upsample2_bwd(a2[k]) for k in range(n)])))
    b = _dyadic(rng, half)
    m = rng.standard_normal((n, D, H, W, C_))
    got = run(3, (D, H, W), a, b, m, out_shape=(n, D, H, W, C_))
    ref = bf16((a + np.stack([OU.avgpool2_bwd(b[k], (D, H, W, C_)) for k in range(n)])) * (bf16(m) > 0))
    assert np.array_equal(got, ref)


def test_head_forward_and_loss_gradients(L):
    import torch
    rng = np.random.default_rng(5)
    nvox = 3000
    d1 = bf16(np.maximum(rng.standard_normal((nvox, 16)), 0.0) * (rng.random((nvox, 16)) < 0.7))
    hw = rng.standard_normal(16).astype(np.float32)
    hb = np.array([0.3], np.float32)
    t = rng.standard_normal(nvox).astype(np.float32)
    out = torch.empty(nvox, device="cuda")
    g_hw = torch.empty(16, device="cuda")
    g_hb = torch.empty(1, device="cuda")
    g_d1 = torch.empty((nvox, 16), device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    L.check(L.lib().unet_head(nvox, ptr(dev(d1)), ptr(dev(hw)), ptr(dev(hb)), ptr(dev(t)), ptr(out), ptr(g_hw),
                              ptr(g_hb), ptr(g_d1), ptr(loss), None), "unet_head")
    ref_out = d1 @ hw.astype(np.float64) + 0.3
    assert rel(out.cpu().numpy(), ref_out) <= TOL
    o = out.cpu().numpy().astype(np.float64)          # the backward pass starts from the GPU's own output
    diff = o - t
    dout = 2.0 * diff / nvox
    assert abs(loss.item() - np.mean(diff ** 2)) <= TOL * np.mean(diff ** 2)
    assert rel(g_hw.cpu().numpy(), dout @ d1) <= TOL
    assert rel(g_hb.cpu().numpy(), [dout.sum()]) <= TOL
    want = dout[:, None] * hw * (d1 > 0)
    got = g_d1.cpu().numpy()
    assert np.all(got[d1 <= 0] == 0)
    mag = np.maximum(np.abs(want), 1e-38)
    ulp = np.exp2(np.floor(np.log2(mag)) - 7)                  # one BF16 unit (8-bit significand) at each value
    assert np.all(np.abs(got - bf16(want)) <= ulp)
    assert np.mean(got != bf16(want)) <= 1e-3

"""tcgen05 3x3x3 convolution (through the C ABI) against the FP64 oracle.

Inputs and weights are BF16-representable, so every product is exact in
FP32 and the only difference from the oracle is the FP32 summation order:
relative L2 error <= 1e-5.
"""
import numpy as np
import pytest

import oracle
from oracle import unet as U

pytestmark = pytest.mark.gpu


def bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


@pytest.fixture(scope="module")
def conv():
    import ctypes as C

    import torch

    import paper_1711_04471_gb300 as P
    P.build()
    from paper_1711_04471_gb300 import _native as N
    L = N.lib()
    oracle.lib()

    def run(x, w, b, epi, mask=None):
        n, D, H, W, cin = x.shape
        cout = w.shape[1]
        xt = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
        wt = torch.from_numpy(np.ascontiguousarray(w, np.float32)).cuda()
        bt = torch.from_numpy(np.ascontiguousarray(b, np.float32)).cuda()
        mt = None if mask is None else torch.from_numpy(np.ascontiguousarray(mask, np.float32)).cuda()
        y = torch.empty((n, D, H, W, cout), dtype=torch.float32, device="cuda")
        st = L.unet_conv3d(n, D, H, W, cin, cout, C.c_void_p(xt.data_ptr()), C.c_void_p(wt.data_ptr()),
                           C.c_void_p(bt.data_ptr()), epi, None if mt is None else C.c_void_p(mt.data_ptr()),
                           C.c_void_p(y.data_ptr()), None)
        N.check(st, "unet_conv3d")
        return y.cpu().numpy()
    return run


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("shape,cin,cout", [((2, 4, 8, 16), 16, 16), ((1, 3, 4, 32), 16, 32), ((1, 2, 2, 128), 32, 64),
                                            ((1, 2, 1, 256), 64, 32), ((2, 5, 8, 16), 64, 16), ((1, 4, 4, 32), 32, 16),
                                            ((1, 3, 8, 16), 16, 64), ((1, 2, 4, 32), 32, 32),
                                            # small planes: tiles of several planes, partial last tiles,
                                            # tiles that cross from one sample into the next
                                            ((3, 2, 4, 4), 32, 64), ((3, 2, 4, 4), 64, 32), ((2, 3, 8, 8), 16, 32),
                                            ((1, 4, 8, 8), 64, 16), ((1, 2, 4, 4), 32, 32), ((2, 4, 4, 8), 32, 16),
                                            ((5, 2, 4, 4), 16, 16)])
def test_conv_forward_bias_relu(conv, shape, cin, cout):
    rng = np.random.default_rng(cin * 100 + cout)
    n, D, H, W = shape
    x = bf16(rng.standard_normal((n, D, H, W, cin)))
    w = bf16(rng.standard_normal((27, cout, cin)) * 0.2)
    b = rng.standard_normal(cout).astype(np.float32)
    y = conv(x, w, b, 0)
    ref = np.stack([np.maximum(U.conv3d(x[k].astype(np.float64), w.astype(np.float64), b.astype(np.float64)), 0)
                    for k in range(n)])
    assert rel(y, ref) <= 1e-5


def test_conv_raw_and_mask_epilogues(conv):
    rng = np.random.default_rng(3)
    x = bf16(rng.standard_normal((2, 4, 4, 32, 32)))
    w = bf16(rng.standard_normal((27, 16, 32)) * 0.2)
    b = np.zeros(16, np.float32)
    raw = np.stack([U.conv3d(x[k].astype(np.float64), w.astype(np.float64)) for k in range(2)])
    assert rel(conv(x, w, b, 1), raw) <= 1e-5
    mask = bf16(rng.standard_normal((2, 4, 4, 32, 16)))
    got = conv(x, w, b, 2, mask)
    assert rel(got, raw * (mask > 0)) <= 1e-5
    assert np.all(got[mask <= 0] == 0)


def test_conv_sample_boundary_in_z(conv):
    """Samples are stacked along z; no tap may read the neighbouring sample."""
    rng = np.random.default_rng(4)
    x = np.zeros((2, 3, 8, 16, 16), np.float32)
    x[1] = bf16(rng.standard_normal((3, 8, 16, 16)))      # sample 0 all zero
    w = bf16(rng.standard_normal((27, 16, 16)))
    y = conv(x, w, np.zeros(16, np.float32), 1)
    assert not np.any(y[0])


def test_conv_epilogues_on_multi_plane_tiles(conv):
    rng = np.random.default_rng(4)
    x = bf16(rng.standard_normal((3, 2, 4, 4, 64)))
    w = bf16(rng.standard_normal((27, 32, 64)) * 0.2)
    b = np.zeros(32, np.float32)
    raw = np.stack([U.conv3d(x[k].astype(np.float64), w.astype(np.float64)) for k in range(3)])
    assert rel(conv(x, w, b, 1), raw) <= 1e-5
    mask = bf16(rng.standard_normal((3, 2, 4, 4, 32)))
    got = conv(x, w, b, 2, mask)
    assert rel(got, raw * (mask > 0)) <= 1e-5
    assert np.all(got[mask <= 0] == 0)

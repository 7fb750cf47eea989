"""FP64 oracle of the warm-start U-Net (test infrastructure).

Wraps the C operators of oracle/unet_oracle.c and composes the network in
numpy.  Architecture (3 levels, 16/32/64 channels, 3x3x3 convolutions with
zero padding, ReLU, 2x2x2 average pooling, nearest-neighbour upsampling,
skip connections by channel concatenation [upsampled, skip]):

    l1a 2->16, l1b 16->16          -> s1          (full resolution)
    pool, l2a 16->32, l2b 32->32   -> s2          (1/2)
    pool, l3a 32->64, l3b 64->32                  (1/4)
    up, cat s2 (64), l2c 64->16                   (1/2)
    up, cat s1 (32), l1c 32->16                   (full)
    head: 1x1x1 16->1, no activation

Two input channels, one output channel; what they hold for the learned
warm start (coarse residual and pressure in, scaled coarse increment out)
is defined in oracle/warmstart.py.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

LAYERS = [("l1a", 2, 16), ("l1b", 16, 16), ("l2a", 16, 32), ("l2b", 32, 32), ("l3a", 32, 64), ("l3b", 64, 32),
          ("l2c", 64, 16), ("l1c", 32, 16)]
HEAD = ("head", 16, 1)

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def declare(L):
    def sig(name, args):
        f = getattr(L, name)
        f.restype = None
        f.argtypes = args
    i = C.c_int
    sig("oracle_conv3d_fwd", [i, i, i, i, i, _dp, _dp, C.c_void_p, _dp])
    sig("oracle_conv3d_bwd_data", [i, i, i, i, i, _dp, _dp, _dp])
    sig("oracle_conv3d_bwd_weight", [i, i, i, i, i, _dp, _dp, _dp, C.c_void_p])
    for n in ("avgpool2_fwd", "avgpool2_bwd", "upsample2_fwd", "upsample2_bwd"):
        sig("oracle_" + n, [i, i, i, i, _dp, _dp])


def _L():
    from . import lib
    return lib()


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def conv3d(x, w, b=None):
    """x (D, H, W, Cin), w (27, Cout, Cin), b (Cout,) -> (D, H, W, Cout)."""
    D, H, W, Cin = x.shape
    Cout = w.shape[1]
    y = np.empty((D, H, W, Cout))
    bb = None if b is None else _c(b)
    _L().oracle_conv3d_fwd(D, H, W, Cin, Cout, _c(x), _c(w), None if bb is None else bb.ctypes.data, y)
    return y


def conv3d_bwd_data(dy, w, Cin):
    D, H, W, Cout = dy.shape
    dx = np.empty((D, H, W, Cin))
    _L().oracle_conv3d_bwd_data(D, H, W, Cin, Cout, _c(dy), _c(w), dx)
    return dx


def conv3d_bwd_weight(x, dy):
    D, H, W, Cin = x.shape
    Cout = dy.shape[3]
    dw = np.empty((27, Cout, Cin))
    db = np.empty(Cout)
    _L().oracle_conv3d_bwd_weight(D, H, W, Cin, Cout, _c(x), _c(dy), dw, db.ctypes.data)
    return dw, db


def avgpool2(x):
    D, H, W, Cc = x.shape
    y = np.empty((D // 2, H // 2, W // 2, Cc))
    _L().oracle_avgpool2_fwd(D, H, W, Cc, _c(x), y)
    return y


def avgpool2_bwd(dy, shape):
    D, H, W, Cc = shape
    dx = np.empty(shape)
    _L().oracle_avgpool2_bwd(D, H, W, Cc, _c(dy), dx)
    return dx


def upsample2(x):
    D, H, W, Cc = x.shape
    y = np.empty((2 * D, 2 * H, 2 * W, Cc))
    _L().oracle_upsample2_fwd(D, H, W, Cc, _c(x), y)
    return y


def upsample2_bwd(dy):
    D2, H2, W2, Cc = dy.shape
    dx = np.empty((D2 // 2, H2 // 2, W2 // 2, Cc))
    _L().oracle_upsample2_bwd(D2 // 2, H2 // 2, W2 // 2, Cc, _c(dy), dx)
    return dx


def init_params(seed=0, scale=1.0):
    """He-normal weights from a numpy generator (oracle-side tests only)."""
    rng = np.random.default_rng(seed)
    P = {}
    for name, ci, co in LAYERS:
        P[name + ".w"] = rng.standard_normal((27, co, ci)) * scale * np.sqrt(2.0 / (27 * ci))
        P[name + ".b"] = rng.standard_normal(co) * 0.01 * scale
    P["head.w"] = rng.standard_normal((1, 16)) * scale * np.sqrt(1.0 / 16)
    P["head.b"] = np.zeros(1)
    return P


def forward(P, x):
    """x (D, H, W, 2) -> (out (D, H, W, 1), cache)."""
    c = {}

    def cr(name, inp):
        z = conv3d(inp, P[name + ".w"], P[name + ".b"])
        a = np.maximum(z, 0.0)
        c[name] = (inp, a)
        return a

    s1 = cr("l1b", cr("l1a", x))
    p1 = avgpool2(s1)
    s2 = cr("l2b", cr("l2a", p1))
    p2 = avgpool2(s2)
    b3 = cr("l3b", cr("l3a", p2))
    u2 = np.concatenate([upsample2(b3), s2], axis=3)
    d2 = cr("l2c", u2)
    u1 = np.concatenate([upsample2(d2), s1], axis=3)
    d1 = cr("l1c", u1)
    out = d1 @ P["head.w"].T + P["head.b"]
    c["shapes"] = (s1.shape, s2.shape, p1.shape, p2.shape)
    c["d1"] = d1
    return out, c


def backward(P, c, dout):
    """Gradients of every parameter for dL/dout."""
    G = {}
    d1 = c["d1"]
    G["head.w"] = np.einsum("zyxo,zyxc->oc", dout, d1)
    G["head.b"] = dout.sum(axis=(0, 1, 2))
    g = dout @ P["head.w"]

    def crb(name, g_out):
        inp, a = c[name]
        gz = g_out * (a > 0)
        dw, db = conv3d_bwd_weight(inp, gz)
        G[name + ".w"], G[name + ".b"] = dw, db
        return conv3d_bwd_data(gz, P[name + ".w"], inp.shape[3])

    gu1 = crb("l1c", g)
    gd2 = upsample2_bwd(gu1[..., :16])
    gs1 = gu1[..., 16:].copy()
    gu2 = crb("l2c", gd2)
    gb3 = upsample2_bwd(gu2[..., :32])
    gs2 = gu2[..., 32:].copy()
    gp2 = crb("l3a", crb("l3b", gb3))
    gs2 = gs2 + avgpool2_bwd(gp2, c["shapes"][1])
    gp1 = crb("l2a", crb("l2b", gs2))
    gs1 = gs1 + avgpool2_bwd(gp1, c["shapes"][0])
    crb("l1a", crb("l1b", gs1))
    return G


def mse(out, target):
    d = out - target
    return float(np.mean(d * d)), 2.0 * d / d.size

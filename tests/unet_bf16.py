"""The warm-start U-Net in FP64 with BF16 rounding at exactly the points
where the GPU network stores BF16 (test helper, not collected).

The arithmetic is the FP64 oracle's (oracle/unet.py: convolutions, their
adjoints, pooling, upsampling); between operators the values are rounded to
BF16 (nearest even, through FP32) wherever the GPU writes a BF16 tensor:
the padded input of l1a, every layer's ReLU output, the pooled maps, and in
the backward pass every gradient tensor handed from one kernel to the next.
Weights enter as BF16 (the GPU's packed weights), biases and the 1x1 head
as FP32.  What remains between this helper and the GPU is the FP32
summation order of the tensor-core accumulations, which can move a stored
value across a BF16 rounding boundary now and then.
"""
import numpy as np

from oracle import unet as OU

LAYERS = OU.LAYERS


def bf16(a):
    """Round to BF16, nearest even (through FP32), returned as FP64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _per_sample(fn, *arrays):
    return np.stack([fn(*(a[k] for a in arrays)) for k in range(arrays[0].shape[0])])


def conv(x, w, b=None):
    return _per_sample(lambda xs: OU.conv3d(xs, w, b), x)


def conv_t(gy, w, cin):
    return _per_sample(lambda g: OU.conv3d_bwd_data(g, w, cin), gy)


def wgrad(x, gy):
    dw, db = 0.0, 0.0
    for k in range(x.shape[0]):
        a, b = OU.conv3d_bwd_weight(x[k], gy[k])
        dw, db = dw + a, db + b
    return dw, db


def pool(x):
    return _per_sample(OU.avgpool2, x)


def pool_adj(g, shape):
    return _per_sample(lambda gs: OU.avgpool2_bwd(gs, shape[1:]), g)


def up(x):
    return _per_sample(OU.upsample2, x)


def up_adj(g):
    return _per_sample(OU.upsample2_bwd, g)


def forward(P, x):
    """x (n, D, H, W, 2) -> (out (n, D, H, W), cache)."""
    c = {}
    relu = lambda z: np.maximum(z, 0.0)

    def layer(name, inp):
        a = bf16(relu(conv(inp, bf16(P[name + ".w"]), P[name + ".b"])))
        c[name] = (inp, a)
        return a

    x16 = bf16(x)
    s1 = layer("l1b", layer("l1a", x16))
    p1 = bf16(pool(s1))
    s2 = layer("l2b", layer("l2a", p1))
    p2 = bf16(pool(s2))
    b3 = layer("l3b", layer("l3a", p2))
    u2 = np.concatenate([up(b3), s2], axis=4)
    d2 = layer("l2c", u2)
    u1 = np.concatenate([up(d2), s1], axis=4)
    d1 = layer("l1c", u1)
    out = (d1 @ np.asarray(P["head.w"], np.float64).T)[..., 0] + float(P["head.b"][0])
    c.update(out=out, d1=d1, s1=s1, s2=s2, p1=p1, p2=p2, u1=u1, u2=u2)
    return out, c


def backward(P, c, target):
    """Loss and gradients of MSE(out, target) in the GPU's storage points."""
    W = {name: bf16(P[name + ".w"]) for name, _, _ in LAYERS}
    out, d1 = c["out"], c["d1"]
    nvox = out.size
    diff = np.float32(out) - np.float32(target)
    loss = float(np.sum(diff.astype(np.float64) ** 2) / nvox)
    dout = (2.0 * diff.astype(np.float64)) / nvox
    G = {"head.w": np.einsum("nzyx,nzyxc->c", dout, d1)[None, :], "head.b": np.array([dout.sum()])}
    hw = np.asarray(P["head.w"], np.float64)[0]
    g_d1 = bf16(dout[..., None] * hw * (d1 > 0))

    def grads(name, gz):
        G[name + ".w"], G[name + ".b"] = wgrad(c[name][0], gz)

    u1, u2, s1, s2 = c["u1"], c["u2"], c["s1"], c["s2"]
    grads("l1c", g_d1)
    g_u1 = bf16(conv_t(g_d1, W["l1c"], 32) * (u1 > 0))
    g_d2 = bf16(up_adj(g_u1[..., :16]))
    grads("l2c", g_d2)
    g_u2 = bf16(conv_t(g_d2, W["l2c"], 64) * (u2 > 0))
    g_b3 = bf16(up_adj(g_u2[..., :32]))
    grads("l3b", g_b3)
    g_a3a = bf16(conv_t(g_b3, W["l3b"], 64) * (c["l3a"][1] > 0))
    grads("l3a", g_a3a)
    g_p2 = bf16(conv_t(g_a3a, W["l3a"], 32))
    g_s2 = bf16((g_u2[..., 32:] + pool_adj(g_p2, s2.shape)) * (s2 > 0))
    grads("l2b", g_s2)
    g_a2a = bf16(conv_t(g_s2, W["l2b"], 32) * (c["l2a"][1] > 0))
    grads("l2a", g_a2a)
    g_p1 = bf16(conv_t(g_a2a, W["l2a"], 16))
    g_s1 = bf16((g_u1[..., 16:] + pool_adj(g_p1, s1.shape)) * (s1 > 0))
    grads("l1b", g_s1)
    g_a1a = bf16(conv_t(g_s1, W["l1b"], 16) * (c["l1a"][1] > 0))
    grads("l1a", g_a1a)
    return loss, G

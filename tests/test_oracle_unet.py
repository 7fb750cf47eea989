"""Pins of the FP64 U-Net operators and of the whole network's gradient."""
import numpy as np
import pytest

import oracle
from oracle import unet as U

oracle.lib()


def offsets(tap):
    return tap // 9 - 1, (tap // 3) % 3 - 1, tap % 3 - 1


def test_conv_impulse_response_and_padding():
    rng = np.random.default_rng(0)
    D, H, W, Cin, Cout = 5, 4, 6, 3, 2
    w = rng.standard_normal((27, Cout, Cin))
    for v in [(2, 1, 3), (0, 0, 0), (4, 3, 5)]:
        x = np.zeros((D, H, W, Cin))
        x[v + (1,)] = 1.0
        y = U.conv3d(x, w)
        seen = np.zeros((D, H, W), bool)
        for tap in range(27):
            dz, dy, dx = offsets(tap)
            u = (v[0] - dz, v[1] - dy, v[2] - dx)
            if 0 <= u[0] < D and 0 <= u[1] < H and 0 <= u[2] < W:
                assert np.array_equal(y[u], w[tap][:, 1])
                seen[u] = True
        assert not np.any(y[~seen])          # nothing leaks through the zero padding


def test_centre_tap_is_a_pointwise_matrix_multiply():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 4, 5, 6))
    w = np.zeros((27, 7, 6))
    w[13] = rng.standard_normal((7, 6))
    b = rng.standard_normal(7)
    assert np.allclose(U.conv3d(x, w, b), np.einsum("zyxc,oc->zyxo", x, w[13]) + b, rtol=1e-13, atol=1e-13)


def test_bwd_data_is_the_adjoint_of_conv():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 5, 3, 4))
    w = rng.standard_normal((27, 6, 4))
    g = rng.standard_normal((4, 5, 3, 6))
    lhs = np.sum(U.conv3d(x, w) * g)
    rhs = np.sum(x * U.conv3d_bwd_data(g, w, 4))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_bwd_weight_by_linearity_in_w():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((3, 4, 5, 2))
    w = rng.standard_normal((27, 3, 2))
    g = rng.standard_normal((3, 4, 5, 3))
    dw, db = U.conv3d_bwd_weight(x, g)
    assert abs(np.sum(dw * w) - np.sum(U.conv3d(x, w) * g)) <= 1e-12 * np.abs(dw).sum() * np.abs(w).max()
    assert np.allclose(db, g.sum(axis=(0, 1, 2)), rtol=1e-14)


def test_pool_and_upsample():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((4, 6, 2, 3))
    assert np.allclose(U.avgpool2(np.ones((4, 4, 4, 2)) * 3.0), 3.0)
    p = U.avgpool2(x)
    g = rng.standard_normal(p.shape)
    assert abs(np.sum(p * g) - np.sum(x * U.avgpool2_bwd(g, x.shape))) < 1e-12
    u = U.upsample2(p)
    assert np.array_equal(u[1::2, ::2, 1::2], p)
    gu = rng.standard_normal(u.shape)
    assert abs(np.sum(u * gu) - np.sum(p * U.upsample2_bwd(gu))) < 1e-12


def test_parameter_count_is_about_200k():
    n = sum(27 * ci * co + co for _, ci, co in U.LAYERS) + 16 + 1
    assert 195_000 < n < 205_000


@pytest.mark.parametrize("seed", [0, 1])
def test_network_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(10 + seed)
    P = U.init_params(seed)
    x = rng.standard_normal((4, 4, 8, 2))
    t = rng.standard_normal((4, 4, 8, 1))
    out, c = U.forward(P, x)
    loss, dout = U.mse(out, t)
    G = U.backward(P, c, dout)
    h = 1e-6
    checked = 0
    for name in sorted(P):
        flat = P[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(3, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = U.mse(U.forward(P, x)[0], t)
            flat[idx] = old - h
            lm, _ = U.mse(U.forward(P, x)[0], t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = G[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1e-3, abs(fd)) + 1e-9, (name, idx, fd, an)
            checked += 1
    assert checked >= 40

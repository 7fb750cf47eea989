"""Pins of the BF16-faithful test helper (tests/unet_bf16.py) on the CPU:
its rounding is the IEEE round-to-nearest-even to an 8-bit significand
(checked against PyTorch's bfloat16 conversion), and with rounding removed
it is the FP64 oracle network itself."""
import numpy as np
import pytest

import oracle
from oracle import unet as OU

import unet_bf16 as UB

oracle.lib()


def test_bf16_rounding_is_round_to_nearest_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 0.0, -0.0, 65504.0]])
    want = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).float().double().numpy()
    assert np.array_equal(UB.bf16(a), want)
    assert UB.bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0            # tie to even
    assert UB.bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6


def test_helper_without_rounding_is_the_oracle_network(monkeypatch):
    rng = np.random.default_rng(1)
    P = OU.init_params(seed=2)
    x = rng.standard_normal((1, 4, 8, 8, 2))
    t = rng.standard_normal((1, 4, 8, 8))
    monkeypatch.setattr(UB, "bf16", lambda a: np.asarray(a, np.float64))
    out, c = UB.forward(P, x)
    ref, rc = OU.forward(P, x[0])
    assert np.abs(out[0] - ref[..., 0]).max() <= 1e-12 * np.abs(ref).max()
    loss, G = UB.backward(P, c, t)
    lo, dout = OU.mse(ref, t[0][..., None])
    Go = OU.backward(P, rc, dout)
    assert abs(loss - lo) <= 1e-6 * lo       # the helper forms out - t in FP32, as the GPU does
    for k in Go:
        assert np.abs(G[k] - Go[k]).max() <= 1e-6 * np.abs(Go[k]).max() + 1e-300, k

"""Host logic of the warm start's training data (CPU tensors): the mixed
batches are linear combinations of solved pairs, renormalised as the
features are, and never pair a residual with its own previous pressure."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1711_04471_gb300 import train_unet as TU


def _data(n=6, shape=(2, 4, 4), seed=0):
    g = torch.Generator().manual_seed(seed)
    r = torch.randn((n,) + shape, generator=g, dtype=torch.float64)
    rms = r.pow(2).mean(dim=(1, 2, 3), keepdim=True).sqrt()
    p = torch.randn((n,) + shape, generator=g, dtype=torch.float64)
    X = torch.stack([r / rms, p], dim=-1).float()
    S = (rms.view(n) * 3.0).float()                     # s = (f dx)^2 rms(r_c) with (f dx)^2 = 3
    T = torch.randn((n,) + shape, generator=g).float()  # any increment: only linearity is checked
    return X, T, S


def test_mixed_batch_is_a_renormalised_linear_combination():
    X, T, S = _data()
    gen = torch.Generator().manual_seed(1)
    ia, ib = torch.tensor([0, 1, 2, 3]), torch.tensor([5, 4, 3, 2])
    x, t = TU.mixed_batch(X, T, S, ia, ib, gen)
    assert x.shape == (4, 2, 4, 4, 2) and t.shape == (4, 2, 4, 4)
    # the residual channel has RMS 1, as warm_start_features makes it
    assert torch.allclose(x[..., 0].pow(2).mean(dim=(1, 2, 3)), torch.ones(4), rtol=1e-5)
    for k in range(4):
        a, b = int(ia[k]), int(ib[k])
        ua, ub = S[a] * X[a, ..., 0], S[b] * X[b, ..., 0]
        va, vb = S[a] * T[a], S[b] * T[b]
        # x0 and t are (alpha ua + beta ub, alpha va + beta vb) / r for one (alpha, beta, r):
        # solve for alpha/r, beta/r from x0 by least squares and check t with them
        A = torch.stack([ua.flatten(), ub.flatten()], 1).double()
        coef = torch.linalg.lstsq(A, x[k, ..., 0].flatten().double().unsqueeze(1)).solution.flatten()
        assert torch.allclose(A @ coef, x[k, ..., 0].flatten().double(), atol=1e-5)
        tv = coef[0] * va.double() + coef[1] * vb.double()
        assert torch.allclose(tv, t[k].double(), atol=1e-4)


def test_single_pairs_keep_their_target_up_to_sign():
    X, T, S = _data()
    gen = torch.Generator().manual_seed(2)
    ia = torch.arange(6)
    x, t = TU.mixed_batch(X, T, S, ia, ia, gen)   # a + b of the same pair is still that pair, rescaled
    for k in range(6):
        sgn = torch.sign((x[k, ..., 0] * X[k, ..., 0]).sum())
        assert torch.allclose(x[k, ..., 0], sgn * X[k, ..., 0], atol=1e-5)
        assert torch.allclose(t[k], sgn * T[k], atol=1e-4)


def test_augment_rolls_and_mirrors_whole_blocks():
    X, T, S = _data(n=2)
    Xa, Ta, Sa = TU.augment(X, T, S)
    assert Xa.shape[0] == 2 * 2 * 4 and Sa.shape == (16,)
    assert torch.equal(Xa[2:4], torch.roll(X, 1, 2))                 # shift by one block in y
    assert torch.equal(Ta[8:10], T.flip(2))                          # mirrored, unshifted

"""The GPU U-Net (tcgen05 convolutions, BF16 activations, FP32 accumulation)
against the FP64 oracle network with the same parameters.

Against the BF16-faithful FP64 network (tests/unet_bf16.py: the oracle's
operators, rounded to BF16 where the GPU stores BF16) the output must agree
to a relative L2 error of 1e-2 and every layer's gradients to 1e-2; only the
FP32 summation order separates the two.  Against the plain FP64 oracle,
which rounds nothing, the BF16 storage of the activations accounts for a
few per cent (output <= 3e-2, gradients aligned).  Training must reduce the
loss; the LES with the network as warm start still converges to the same
tolerance (the solve decides the answer).
"""
import numpy as np
import pytest

import oracle
from oracle import unet as OU

import unet_bf16 as UB

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def U():
    import paper_1711_04471_gb300 as P
    P.build()
    from paper_1711_04471_gb300 import unet
    oracle.lib()
    return unet


def bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


def sample(rng, n, D, H, W):
    x = bf16(rng.standard_normal((n, D, H, W, 2)))
    t = rng.standard_normal((n, D, H, W)).astype(np.float32) * 0.5
    return x, t


def test_forward_matches_oracle(U):
    import torch
    rng = np.random.default_rng(0)
    x, _ = sample(rng, 2, 4, 32, 64)
    with U.UNet(seed=3) as net:
        P = U.unflatten(bf16(net.get_params()).astype(np.float64))
        net.set_params(U.flatten(P))
        y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    want, _ = UB.forward(P, x.astype(np.float64))
    err = np.linalg.norm(y - want) / np.linalg.norm(want)
    print(f"network output vs BF16-faithful FP64 network: rel-L2 {err:.2e}")
    assert err <= 1e-2, err
    for k in range(2):
        ref, _ = OU.forward(P, x[k].astype(np.float64))
        assert np.linalg.norm(y[k] - ref[..., 0]) / np.linalg.norm(ref) <= 3e-2


@pytest.mark.parametrize("shape", [(1, 4, 32, 64), (4, 8, 16, 16)])
def test_gradients_match_oracle(U, shape):
    """Every layer's weight and bias gradients (tcgen05 weight gradients,
    backward-data with flipped weights) against the BF16-faithful FP64
    network at 1e-2 relative; the second shape is the warm-start training
    batch geometry (coarse 8 x 16 x 16 grids: multi-plane tiles at the
    coarse levels, tiles that cross samples)."""
    import torch
    rng = np.random.default_rng(1)
    x, t = sample(rng, *shape)
    with U.UNet(seed=5) as net:
        P = U.unflatten(bf16(net.get_params()).astype(np.float64))
        net.set_params(U.flatten(P))
        loss, g = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    _, c = UB.forward(P, x.astype(np.float64))
    lo, Gb = UB.backward(P, c, t.astype(np.float64))
    assert abs(loss - lo) <= 1e-2 * lo
    Gg = U.unflatten(g.astype(np.float64))
    errs = {}
    for name in Gb:
        a, b = Gg[name].ravel(), np.asarray(Gb[name]).ravel()
        errs[name] = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-300)
    print("per-layer gradient rel-L2 vs BF16-faithful FP64 network: " +
          " ".join(f"{k} {v:.1e}" for k, v in errs.items()))
    for name, r in errs.items():
        assert r <= 1e-2, (name, r)
    # and against the plain FP64 oracle, which stores nothing in BF16
    if shape[0] == 1:
        out, co = OU.forward(P, x[0].astype(np.float64))
        lo64, dout = OU.mse(out, t[0][..., None].astype(np.float64))
        Go = OU.backward(P, co, dout)
        for name in Go:
            a, b = Gg[name].ravel(), Go[name].ravel()
            cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300)
            assert cos >= 0.99, (name, cos)


def test_training_reduces_loss(U):
    import torch
    rng = np.random.default_rng(2)
    x = torch.from_numpy(bf16(rng.standard_normal((2, 8, 32, 64, 2)))).cuda()
    # a smooth target that depends on the input: a blurred copy of channel 0
    xc = x[..., 0]
    t = (xc + torch.roll(xc, 1, 3) + torch.roll(xc, -1, 3) + torch.roll(xc, 1, 2) + torch.roll(xc, -1, 2)) / 5.0
    t = t.contiguous()
    with U.UNet(seed=7) as net:
        losses = [net.train_step(x, t, 2e-3) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])


def test_les_with_learned_warm_start_converges(U):
    from paper_1711_04471_gb300 import inputs
    from paper_1711_04471_gb300.les import LES
    nx, ny, nz = 64, 32, 16
    solid = inputs.les_buildings(nx, ny, nz, dx=4.0, seed=11, margin_cells=4)
    with U.UNet(seed=1) as net, LES(nx, ny, nz, solid) as plain, LES(nx, ny, nz, solid) as warm:
        warm.set_warm_start(net)
        sp = plain.step(3)
        sw = warm.step(3)
        for a in sw:
            assert a["status"] == 0 and a["rel_res"] <= 1e-6 and a["ms_guess"] > 0
        # both solves reach the tolerance, so the pressures agree to it
        pa, pb = plain.get("p")[1:-1, 1:-1, 1:-1], warm.get("p")[1:-1, 1:-1, 1:-1]
        assert np.linalg.norm(pa - pb) / np.linalg.norm(pa) < 1e-3
        warm.set_warm_start(None)
        assert warm.step(1)[0]["ms_guess"] < 0.05


def test_trained_warm_start_saves_sor_iterations(U):
    """The committed weights on the 256 x 256 x 128 workload (building seed
    1003, which no training run used): from the same states, SOR started
    from the network's guess reaches the same 1e-6 residual in clearly fewer
    iterations than SOR started from the previous pressure."""
    import os

    from paper_1711_04471_gb300 import train_unet
    weights = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                           "paper_1711_04471_gb300", "data", "unet_warmstart.npy")
    with U.UNet(seed=0) as net:
        net.set_params(np.load(weights))
        rows = train_unet.compare_warm_starts(net, spinup=20, steps=3, spinup_tol=1e-4, log=lambda *a: None,
                                              check_every=50, max_iter=400000)
    for r in rows:
        assert r["plain_res"] <= 1e-6 and r["nn_res"] <= 1e-6
    plain = sum(r["plain_iters"] for r in rows)
    nn = sum(r["nn_iters"] for r in rows)
    print(f"SOR iterations over 3 steps: previous-pressure warm start {plain}, learned {nn}")
    assert nn <= 0.6 * plain, (plain, nn)

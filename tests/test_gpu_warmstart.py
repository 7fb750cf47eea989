"""The coarse-grid warm start on the GPU against the FP64 oracle
(oracle/warmstart.py): features (restricted residual and pressure, scale),
the prolongated update, the network on the coarse geometries (tiles that
span several small planes) and its use inside the LES step.

Tolerances: the transfers run in FP64 on the GPU, so the scale and the
update agree to 1e-12 relative (only the summation order differs); the
features are stored in FP32 (1e-6 of their RMS of 1)."""
import numpy as np
import pytest

import oracle
from oracle import les as ol
from oracle import unet as OU
from oracle import warmstart as ows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1711_04471_gb300 as P
    P.build()
    from paper_1711_04471_gb300 import les, unet
    oracle.lib()
    return les, unet


def padded(a):
    out = np.zeros(tuple(n + 2 for n in a.shape))
    out[1:-1, 1:-1, 1:-1] = a
    return out


def fields(rng, nz, ny, nx):
    # a smooth pressure plus noise, and a right-hand side of the same order as A p
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    p = np.cos(np.pi * (x + 0.5) / (2 * nx)) * 50.0 + rng.standard_normal((nz, ny, nx))
    b = (rng.standard_normal((nz, ny, nx)) * 0.1).astype(np.float32)
    return p, b


@pytest.mark.parametrize("f", [1, 2, 4, 8, 16])
def test_features_match_oracle(lib, f):
    import torch
    les, _ = lib
    nz, ny, nx, dx = 32, 48, 64, 4.0
    rng = np.random.default_rng(f)
    p, b = fields(rng, nz, ny, nx)
    x, s = les.warm_start_features(torch.from_numpy(p).cuda(), torch.from_numpy(b).cuda(), dx, f)
    P = ol.make_params(nx, ny, nz, dx=dx)
    xo, so = ows.features(P, padded(b.astype(np.float64)), padded(p), f)
    assert s == pytest.approx(so, rel=1e-12)
    assert np.abs(x.cpu().numpy() - xo).max() <= 1e-6 * max(1.0, np.abs(xo).max())


@pytest.mark.parametrize("f", [1, 2, 8])
def test_apply_matches_oracle(lib, f):
    import torch
    les, _ = lib
    nz, ny, nx = 16, 24, 32
    rng = np.random.default_rng(10 + f)
    p = rng.standard_normal((nz, ny, nx))
    out = rng.standard_normal((nz // f, ny // f, nx // f)).astype(np.float32)
    s = 0.731
    pt = torch.from_numpy(p.copy()).cuda()
    les.warm_start_apply(torch.from_numpy(out).cuda(), s, pt, f)
    want = ows.apply(padded(p), out.astype(np.float64), s, f)[1:-1, 1:-1, 1:-1]
    assert np.abs(pt.cpu().numpy() - want).max() <= 1e-12 * np.abs(want).max()


def test_zero_residual_gives_zero_scale_and_no_update(lib):
    """p solving A p = b exactly (b formed from p in FP64, then rounded to FP32
    only where exactly representable): the residual is at rounding level."""
    import torch
    les, _ = lib
    nz, ny, nx, dx, f = 16, 16, 32, 4.0, 4
    rng = np.random.default_rng(20)
    p = np.round(rng.standard_normal((nz, ny, nx)) * 64) / 64       # multiples of 1/64: A p exact in FP32
    P = ol.make_params(nx, ny, nz, dx=dx)
    b = ol.interior(ol.apply_A(P, padded(p))).astype(np.float32)
    assert np.array_equal(b.astype(np.float64), ol.interior(ol.apply_A(P, padded(p))))
    x, s = les.warm_start_features(torch.from_numpy(p).cuda(), torch.from_numpy(b).cuda(), dx, f)
    assert s == 0.0
    assert np.all(x.cpu().numpy()[..., 0] == 0)


def bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(torch.bfloat16).float().numpy()


@pytest.mark.parametrize("n", [1, 3])
def test_network_on_the_coarse_grid_matches_oracle(lib, n):
    """16 x 16 x 8: level planes of 256, 64 and 16 voxels; the two lower
    levels use tiles of 2 and 8 planes (crossing samples when n > 1)."""
    import torch
    _, U = lib
    rng = np.random.default_rng(30 + n)
    x = bf16(rng.standard_normal((n, 8, 16, 16, 2)))
    t = (rng.standard_normal((n, 8, 16, 16)) * 0.5).astype(np.float32)
    with U.UNet(seed=4) as net:
        P = U.unflatten(bf16(net.get_params()).astype(np.float64))
        net.set_params(U.flatten(P))
        y = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
        loss, g = net.gradients(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda())
    Gsum, lsum = None, 0.0
    for k in range(n):
        ref, c = OU.forward(P, x[k].astype(np.float64))
        assert np.linalg.norm(y[k] - ref[..., 0]) / np.linalg.norm(ref) <= 3e-2
        lo, dout = OU.mse(ref, t[k][..., None].astype(np.float64))
        Go = OU.backward(P, c, dout)
        lsum += lo
        Gsum = Go if Gsum is None else {a: Gsum[a] + Go[a] for a in Go}
    # the GPU loss and gradients are those of the batch mean
    assert abs(loss - lsum / n) <= 3e-2 * lsum / n
    Gg = U.unflatten(g.astype(np.float64))
    for name in Gsum:
        a, b = Gg[name].ravel(), Gsum[name].ravel() / n
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300)
        assert cos >= 0.99, (name, cos)


def test_les_coarse_warm_start_converges_to_the_plain_solution(lib):
    les, U = lib
    from paper_1711_04471_gb300 import inputs
    nx, ny, nz = 64, 64, 32
    solid = inputs.les_buildings(nx, ny, nz, dx=4.0, seed=12, margin_cells=4)
    with U.UNet(seed=2) as net, les.LES(nx, ny, nz, solid) as plain, les.LES(nx, ny, nz, solid) as warm:
        warm.set_warm_start(net, factor=4)               # coarse grid 16 x 16 x 8
        sp = plain.step(3)
        sw = warm.step(3)
        for a in sw:
            assert a["status"] == 0 and a["rel_res"] <= 1e-6 and a["ms_guess"] > 0
        pa, pb = plain.get("p")[1:-1, 1:-1, 1:-1], warm.get("p")[1:-1, 1:-1, 1:-1]
        assert np.linalg.norm(pa - pb) / np.linalg.norm(pa) < 1e-3
        ua, ub = plain.get("u")[1:-1, 1:-1, 1:-1], warm.get("u")[1:-1, 1:-1, 1:-1]
        assert np.linalg.norm(ua - ub) / np.linalg.norm(ua) < 1e-4
        assert len(sp) == 3


def test_warm_start_factor_is_validated(lib):
    les, U = lib
    with U.UNet(seed=0) as net, les.LES(64, 32, 16) as g:
        with pytest.raises(RuntimeError):
            g.set_warm_start(net, factor=3)
        with pytest.raises(RuntimeError):
            g.set_warm_start(net, factor=8)              # 8 x 4 x 2 coarse grid: too small to pool twice
        g.set_warm_start(net, factor=2)

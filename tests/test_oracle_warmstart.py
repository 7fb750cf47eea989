"""Pins of the warm start's grid transfers in the oracle (oracle/warmstart.py):
brute-force block means, a library trilinear interpolation, exactness on
linear fields, full weighting as the column-by-column adjoint of the
prolongation, the telescoping identity of the Poisson residual, scale
covariance, second-order accuracy of restrict-then-prolong on the slowest
SOR mode and of the full-weighted projection on it."""
import math

import numpy as np
import pytest

from oracle import les as ol
from oracle import warmstart as ws


def _rng(seed):
    return np.random.default_rng(seed)


def test_restrict_is_the_block_mean():
    a = _rng(0).standard_normal((6, 4, 10))
    f = 2
    want = np.zeros((3, 2, 5))
    for K in range(3):
        for J in range(2):
            for I in range(5):
                s = 0.0
                for k in range(f):
                    for j in range(f):
                        for i in range(f):
                            s += a[K * f + k, J * f + j, I * f + i]
                want[K, J, I] = s / f ** 3
    assert np.allclose(ws.restrict(a, f), want, rtol=0, atol=1e-14)
    assert np.array_equal(ws.restrict(a, 1), a)
    with pytest.raises(ValueError):
        ws.restrict(a, 4)


def test_prolong_keeps_constants_away_from_the_outflow_and_is_the_identity_at_f1():
    c = np.full((2, 3, 4), 2.5)
    for f in (1, 2, 4):
        fine = ws.prolong(c, f)
        keep = (np.arange(4 * f) + 0.5) / f - 0.5 <= 3    # up to the last coarse centre
        assert np.allclose(fine[:, :, keep], 2.5, rtol=0, atol=1e-14)
        # past the last centre the value falls linearly to 0 on the outflow face
        x_face = 4 * f
        xs = np.arange(4 * f)[~keep] + 0.5
        assert np.allclose(fine[0, 0, ~keep], 2.5 * (x_face - xs) / (f / 2), rtol=0, atol=1e-13)
    r = _rng(1).standard_normal((3, 4, 5))
    assert np.allclose(ws.prolong(r, 1), r, rtol=0, atol=1e-15)


def test_prolong_matches_library_trilinear_on_a_ghost_padded_field():
    """One ghost coarse cell on every side (mirror in z and at the inflow,
    wrap in y, minus the last value past the outflow), then the library's
    trilinear interpolation of cell-centred data, cropped to the grid."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    c = _rng(2).standard_normal((3, 4, 5))
    f = 4
    t = torch.from_numpy(c)[None, None]
    t = torch.cat([t[:, :, :1], t, t[:, :, -1:]], dim=2)
    t = torch.cat([t[:, :, :, -1:], t, t[:, :, :, :1]], dim=3)
    t = torch.cat([t[..., :1], t, -t[..., -1:]], dim=4)
    up = F.interpolate(t, scale_factor=f, mode="trilinear", align_corners=False)[0, 0].numpy()
    want = up[f:f + 3 * f, f:f + 4 * f, f:f + 5 * f]
    assert np.allclose(ws.prolong(c, f), want, rtol=0, atol=1e-13)


def test_prolong_is_exact_for_fields_linear_in_x_and_z():
    ncz, ncy, ncx, f = 3, 2, 5, 4
    K, J, I = np.meshgrid(np.arange(ncz), np.arange(ncy), np.arange(ncx), indexing="ij")
    c = 2.0 * I - 0.75 * K + 0.5
    fine = ws.prolong(c, f)
    X = (np.arange(ncx * f) + 0.5) / f - 0.5
    Z = (np.arange(ncz * f) + 0.5) / f - 0.5
    want = 2.0 * X[None, None, :] - 0.75 * Z[:, None, None] + 0.5
    inside = ((X >= 0) & (X <= ncx - 1))[None, None, :] & ((Z >= 0) & (Z <= ncz - 1))[:, None, None]
    inside = np.broadcast_to(inside, fine.shape)
    assert np.allclose(fine[inside], np.broadcast_to(want, fine.shape)[inside], rtol=0, atol=1e-13)


def test_residual_sum_telescopes_to_the_outflow_column():
    """Summed over the grid, the 7-point operator leaves only the outflow
    face term (Neumann and periodic fluxes cancel): sum(A p) dx^2 =
    -2 sum over j, k of p(nx, j, k).  Hence sum r = sum b + 2/dx^2 sum p(nx)."""
    nx, ny, nz, dx, f = 8, 6, 4, 4.0, 2
    P = ol.make_params(nx, ny, nz, dx=dx)
    rng = _rng(3)
    b, p = ol.padded(P), ol.padded(P)
    ol.interior(b)[:] = rng.standard_normal((nz, ny, nx))
    ol.interior(p)[:] = rng.standard_normal((nz, ny, nx))
    r = ws.residual_field(P, b, p)
    want = ol.interior(b).sum() + 2.0 / dx ** 2 * p[1:-1, 1:-1, nx].sum()
    assert r.sum() == pytest.approx(want, rel=1e-12, abs=1e-12)
    assert ws.restrict(r, f).sum() * f ** 3 == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_full_weighting_is_the_adjoint_of_prolong():
    """Column by column: restrict_fw(a)[I] = <prolong(e_I), a> / f^3, with e_I
    the coarse unit fields; hence <prolong(c), a> = f^3 <c, restrict_fw(a)>."""
    f, shape_c = 2, (2, 3, 4)
    a = _rng(6).standard_normal(tuple(n * f for n in shape_c))
    got = ws.restrict_fw(a, f)
    for idx in np.ndindex(shape_c):
        e = np.zeros(shape_c)
        e[idx] = 1.0
        assert got[idx] == pytest.approx(np.sum(ws.prolong(e, f) * a) / f ** 3, rel=1e-12, abs=1e-14)
    c = _rng(7).standard_normal(shape_c)
    assert np.sum(ws.prolong(c, f) * a) == pytest.approx(f ** 3 * np.sum(c * got), rel=1e-12)
    assert np.allclose(ws.restrict_fw(a, 1), a, rtol=0, atol=1e-15)


def test_full_weighting_keeps_the_slow_mode_projection():
    """<phi, r> for the slowest mode phi and a rough r: full weighting keeps it
    to O((f/nx)^2) of |phi| |r|; block means make an O(f/nx) error."""
    nx, ny, nz, f = 128, 8, 8, 8
    x = np.arange(nx) + 0.5
    phi = np.broadcast_to(np.cos(np.pi * x / (2 * nx))[None, None, :], (nz, ny, nx))
    phic = np.cos(np.pi * (np.arange(nx // f) + 0.5) * f / (2 * nx))
    worst_fw, worst_bm = 0.0, 0.0
    for seed in range(5):
        r = _rng(10 + seed).standard_normal((nz, ny, nx))
        exact = np.sum(phi * r)
        fw = f ** 3 * np.sum(phic[None, None, :] * ws.restrict_fw(r, f))
        bm = f ** 3 * np.sum(phic[None, None, :] * ws.restrict(r, f))
        scale = np.linalg.norm(phi) * np.linalg.norm(r)
        worst_fw = max(worst_fw, abs(fw - exact) / scale)
        worst_bm = max(worst_bm, abs(bm - exact) / scale)
    assert worst_fw < 3e-3
    assert worst_bm > 3 * worst_fw


def test_features_scale_with_the_fields():
    nx, ny, nz, dx, f = 8, 8, 4, 2.0, 2
    P = ol.make_params(nx, ny, nz, dx=dx)
    rng = _rng(4)
    b, p = ol.padded(P), ol.padded(P)
    ol.interior(b)[:] = rng.standard_normal((nz, ny, nx))
    ol.interior(p)[:] = rng.standard_normal((nz, ny, nx))
    x1, s1 = ws.features(P, b, p, f)
    x2, s2 = ws.features(P, 3.0 * b, 3.0 * p, f)
    assert np.allclose(x1, x2, rtol=1e-12, atol=1e-12)
    assert s2 == pytest.approx(3.0 * s1, rel=1e-12)
    rc = ws.restrict_fw(ws.residual_field(P, b, p), f)
    assert s1 == pytest.approx((f * dx) ** 2 * math.sqrt(np.mean(rc ** 2)), rel=1e-12)
    assert np.mean(x1[..., 0] ** 2) == pytest.approx(1.0, rel=1e-12)
    assert np.mean(x1[..., 1] ** 2) == pytest.approx(1.0, rel=1e-12)


def test_target_then_apply_returns_the_new_pressure_at_f1():
    nx, ny, nz = 6, 4, 4
    P = ol.make_params(nx, ny, nz)
    rng = _rng(5)
    p0, p1 = ol.padded(P), ol.padded(P)
    ol.interior(p0)[:] = rng.standard_normal((nz, ny, nx))
    ol.interior(p1)[:] = rng.standard_normal((nz, ny, nx))
    s = 0.37
    g = ws.apply(p0, ws.target(p0, p1, 1, s), s, 1)
    assert np.allclose(ol.interior(g), ol.interior(p1), rtol=0, atol=1e-14)


def test_coarse_transfer_is_second_order_on_the_slowest_sor_mode():
    """The slowest mode of the solve, cos(pi (i - 1/2) / (2 nx)) along x and
    constant over y-z planes, survives restrict-then-prolong to O((f/nx)^2);
    a half-cell shift in either transfer would leave an O(f/nx) error."""
    nx, ny, nz, f = 128, 8, 8, 8
    x = np.arange(1, nx + 1) - 0.5
    mode = np.broadcast_to(np.cos(np.pi * x / (2 * nx))[None, None, :], (nz, ny, nx))
    back = ws.prolong(ws.restrict(mode, f), f)
    err = np.linalg.norm(back - mode) / np.linalg.norm(mode)
    assert err < 2e-3
    shifted = np.roll(back, 1, axis=2)
    assert np.linalg.norm(shifted - mode) / np.linalg.norm(mode) > 5 * err

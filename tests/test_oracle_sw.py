"""Pins of the FP64 2DSW oracle against what physics and mathematics fix.

None of these compare the oracle with itself: each checks a property that a
dropped term, a wrong sign, a wrong index or a transposed operand in
oracle/sw_oracle.c would break.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1711_04471_gb300 import inputs


def _state(inp):
    return oracle.SWState(inp.params(), inp.H, inp.eta0)


def _lake_at_rest(inp):
    eta = np.maximum(0.0, -inp.H)
    return inputs.SWInput(inp.nx, inp.ny, inp.dx, inp.dy, inp.dt, inp.H, eta, hmin=inp.hmin)


def test_lake_at_rest_is_bit_identical():
    """Still water over any bathymetry (with dry land) must not move at all."""
    base = inputs.sw_wetdry(n=64, seed=7)
    inp = _lake_at_rest(base)
    s = _state(inp)
    eta0 = s.eta.copy()
    s.run(1000)
    assert np.array_equal(s.eta, eta0)
    assert not np.any(s.u) and not np.any(s.v)
    assert 0.0 < s.wet_i.mean() < 1.0


@pytest.mark.parametrize("case", ["hump", "wetdry"])
def test_volume_conserved(case):
    """Face fluxes telescope, wall faces carry nothing and the masked filter
    exchange is antisymmetric, so total volume is conserved to rounding."""
    inp = inputs.sw_hump() if case == "hump" else inputs.sw_wetdry(n=64, seed=11)
    s = _state(inp)
    v0, _ = s.volume()
    s.run(1000)
    v1, _ = s.volume()
    assert abs(v1 - v0) / v0 <= 1e-12
    if case == "wetdry":
        w = s.wet_i.mean()
        assert 0.05 < w < 0.99
        assert np.any(s.u) and np.any(s.v)


def _mode_matrix(kx, ky, dx, dy, dt, g, H, eps):
    """Exact linear map of one step for the mode
    eta = A cos(kx x) cos(ky y), u = Bu sin(kx x) cos(ky y), v = Bv cos(kx x) sin(ky y),
    derived by hand from the scheme's difference operators on that mode."""
    sx = 2.0 * math.sin(kx * dx / 2) / dx
    sy = 2.0 * math.sin(ky * dy / 2) / dy
    r = 1.0 - eps * (math.sin(kx * dx / 2) ** 2 + math.sin(ky * dy / 2) ** 2)
    # momentum: B' = B + g dt s A
    Mb = np.array([[1.0, 0.0, 0.0], [g * dt * sx, 1.0, 0.0], [g * dt * sy, 0.0, 1.0]])
    # continuity then filter: A' = r (A - H dt (sx Bu' + sy Bv'))
    Ma = np.array([[r, -r * H * dt * sx, -r * H * dt * sy], [0, 1, 0], [0, 0, 1]])
    return Ma @ Mb, r


def _fourier_run(a, mx, my, n=32, nsteps=100, H=10.0, dx=10.0, dt=0.1, eps=0.05):
    L = n * dx
    kx, ky = math.pi * mx / L, math.pi * my / L
    xc = (np.arange(n) + 0.5) * dx
    xf = np.arange(n + 1) * dx
    eta0 = a * np.outer(np.cos(ky * xc), np.cos(kx * xc))
    inp = inputs.SWInput(n, n, dx, dx, dt, np.full((n, n), H), eta0)
    s = _state(inp).run(nsteps)
    M, r = _mode_matrix(kx, ky, dx, dx, dt, 9.81, H, eps)
    amp = np.linalg.matrix_power(M, nsteps) @ np.array([a, 0.0, 0.0])
    eta_x = amp[0] * np.outer(np.cos(ky * xc), np.cos(kx * xc))
    u_x = amp[1] * np.outer(np.cos(ky * xc), np.sin(kx * xf))
    v_x = amp[2] * np.outer(np.sin(ky * xf), np.cos(kx * xc))
    scale = np.abs(amp).max()
    err = max(np.abs(s.eta_i - eta_x).max() / a,
              np.abs(s.u_f - u_x).max() / max(abs(amp[1]), 1e-300) if mx else 0.0,
              np.abs(s.v_f - v_x).max() / max(abs(amp[2]), 1e-300) if my else 0.0)
    return err, M, r, scale


@pytest.mark.parametrize("mx,my", [(2, 0), (0, 3), (2, 1), (5, 4)])
def test_linear_fourier_mode_closed_form(mx, my):
    """A small-amplitude standing mode of a flat closed basin follows M^n exactly
    (walls included); the residual mismatch is the O(a/H) nonlinearity, so it
    must shrink in proportion to the amplitude."""
    e6, M, r, _ = _fourier_run(1e-6, mx, my)
    e7, _, _, _ = _fourier_run(1e-7, mx, my)
    assert e7 <= 1e-6, e7
    assert e6 <= 1e-5, e6
    assert 5.0 < e6 / max(e7, 1e-300) < 20.0 or e6 < 1e-9
    assert abs(np.linalg.det(M) - r) < 1e-14


def test_mode_matrix_phase_speed_is_sqrt_gH():
    """The mode matrix itself: in the long-wave, unfiltered limit the phase
    advance per step tends to dt*sqrt(gH)*|k| (gravity waves at sqrt(gH))."""
    g, H, dx, dt = 9.81, 10.0, 10.0, 0.1
    for k in [1e-3, 3e-3]:
        M, r = _mode_matrix(k, 0.0, dx, dx, dt, g, H, 0.0)
        ev = np.linalg.eigvals(M[:2, :2])
        phase = np.abs(np.angle(ev)).max()
        assert abs(phase / (dt * math.sqrt(g * H) * k) - 1.0) < 1e-3


def test_hump_symmetry():
    """The centred hump in a square basin keeps both mirror symmetries and the
    diagonal (transpose) symmetry."""
    s = _state(inputs.sw_hump()).run(1000)
    e = s.eta_i
    tol = 1e-13 * np.abs(e).max() + 1e-15
    assert np.abs(e - e[:, ::-1]).max() <= tol
    assert np.abs(e - e[::-1, :]).max() <= tol
    assert np.abs(e - e.T).max() <= tol
    u, v = s.u_f, s.v_f
    assert np.abs(u - v.T).max() <= 1e-13 * np.abs(u).max()
    assert np.abs(u + u[:, ::-1]).max() <= 1e-13 * np.abs(u).max()


def _crest_radius(s, nx, dx):
    row = 0.5 * (s.eta_i[nx // 2 - 1, :] + s.eta_i[nx // 2, :])
    xc = (np.arange(nx) + 0.5) * dx - nx * dx / 2
    k = int(np.argmax(np.where(xc > 5 * dx, row, -np.inf)))
    y0, y1, y2 = row[k - 1], row[k], row[k + 1]
    return xc[k] + 0.5 * (y0 - y2) / (y0 - 2 * y1 + y2) * dx


def test_hump_front_travels_at_sqrt_gH():
    """Config-1 geometry with a small (linear) hump: the ring crest moves at
    sqrt(gH) = 9.9 m/s between t = 20 s and t = 30 s (the crest's offset from
    r = ct, of order sigma, cancels in the difference)."""
    inp = inputs.sw_hump(amp=0.01)
    r = []
    for steps in (200, 300):
        s = _state(inp).run(steps)
        r.append(_crest_radius(s, inp.nx, inp.dx))
    speed = (r[1] - r[0]) / (100 * inp.dt)
    assert abs(speed / math.sqrt(9.81 * 10.0) - 1.0) < 0.02, speed


# ---------------------------------------------------------------------------
# Brute force: an independent per-face transcription of the scheme on 8x8,
# using dictionaries keyed by cell and face, no arrays.
# ---------------------------------------------------------------------------

def _brute_force(H, eta0, dx, dy, dt, g, eps, hmin, nsteps):
    ny, nx = H.shape
    eta = {(i, j): float(eta0[j - 1, i - 1]) for i in range(1, nx + 1) for j in range(1, ny + 1)}
    dep = {(i, j): float(H[j - 1, i - 1]) for i in range(1, nx + 1) for j in range(1, ny + 1)}
    # faces: ('x', i, j) between (i,j) and (i+1,j); ('y', i, j) between (i,j) and (i,j+1)
    faces = [('x', i, j) for j in range(1, ny + 1) for i in range(0, nx + 1)] + \
            [('y', i, j) for i in range(1, nx + 1) for j in range(0, ny + 1)]
    vel = {f: 0.0 for f in faces}

    def cells_of(f):
        k, i, j = f
        return ((i, j), (i + 1, j)) if k == 'x' else ((i, j), (i, j + 1))

    for _ in range(nsteps):
        depth = {c: dep[c] + eta[c] for c in eta}
        wet = {c: depth[c] > hmin for c in eta}
        new_vel = {}
        for f in faces:
            a, b = cells_of(f)
            if a not in eta or b not in eta:        # wall face
                new_vel[f] = 0.0
                continue
            d = dx if f[0] == 'x' else dy
            w = vel[f] - g * dt * (eta[b] - eta[a]) / d
            ok = (wet[a] and wet[b]) or (wet[a] and w > 0) or (wet[b] and w < 0)
            new_vel[f] = w if ok else 0.0
        div = {c: 0.0 for c in eta}
        for f in faces:
            a, b = cells_of(f)
            w = new_vel[f]
            if w == 0.0:
                continue
            d = dx if f[0] == 'x' else dy
            flux = w * (depth[a] if w > 0 else depth[b]) / d
            if a in div:
                div[a] += flux
            if b in div:
                div[b] -= flux
        star = {c: eta[c] - dt * div[c] for c in eta}
        out = {}
        for (i, j) in eta:
            if not wet[(i, j)]:
                out[(i, j)] = star[(i, j)]
                continue
            nbs = [n for n in ((i + 1, j), (i - 1, j), (i, j + 1), (i, j - 1)) if n in eta and wet[n]]
            out[(i, j)] = star[(i, j)] + eps / 4 * sum(star[n] - star[(i, j)] for n in nbs)
        eta, vel = out, new_vel
    E = np.array([[eta[(i, j)] for i in range(1, nx + 1)] for j in range(1, ny + 1)])
    U = np.array([[vel[('x', i, j)] for i in range(0, nx + 1)] for j in range(1, ny + 1)])
    V = np.array([[vel[('y', i, j)] for i in range(1, nx + 1)] for j in range(0, ny + 1)])
    return E, U, V


@pytest.mark.parametrize("seed", [3, 5, 8])
def test_brute_force_8x8(seed):
    rng = inputs.SplitMix64(seed)
    n = 8
    H = rng.uniform(n * n, -1.0, 3.0).reshape(n, n)
    eta_init = rng.uniform(n * n, -0.3, 0.3).reshape(n, n)
    eta0 = np.maximum(eta_init, -H)
    inp = inputs.SWInput(n, n, 10.0, 8.0, 0.2, H, eta0)
    s = _state(inp).run(50)
    E, U, V = _brute_force(H, eta0, 10.0, 8.0, 0.2, 9.81, 0.05, 0.05, 50)
    assert s.margin > 1e-6
    assert np.abs(s.eta_i - E).max() <= 1e-14 * max(1.0, np.abs(E).max()) * 50
    assert np.abs(s.u_f - U).max() <= 1e-13
    assert np.abs(s.v_f - V).max() <= 1e-13
    assert 0 < s.wet_i.sum() < n * n

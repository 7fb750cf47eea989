"""Seeded synthetic inputs for the shallow-water and urban-LES workloads.

This module is shared by the FP64 oracle tests and the CUDA path: it only
*draws* initial states and geometry (bathymetry, surface perturbations,
building masks) and holds none of the time-stepping arithmetic.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then the published 64-bit finaliser.  Uniform doubles take the top 53 bits.

Workloads (the paper's own inputs -- the textbook basin of the 2-D shallow
water model, Sec. 6.2, and the GIS building data and mesoscale forcing of
UFLES, Sec. 6.3 -- are not available; these recipes stand in for them):

* ``sw_hump``      flat 10 m basin, 1 m Gaussian hump of sigma 5 cells at the
                   geometric centre (100 x 100 cells, dx = 10 m).
* ``sw_wetdry``    50 m mean depth minus 32 Gaussian hills of 60 m, widths
                   scaled by bisection so 15 % +- 0.5 % of cells are dry,
                   plus a random-phase 0.5 m surface perturbation.
* ``sw_ensemble``  512 square instances with side log-uniform in [64, 1024].
* ``les_buildings`` random rectangular blocks covering >= 20 % of the ground.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1


class SplitMix64:
    """Counter-based SplitMix64 stream.  ``next_u64(n)`` returns the next n outputs."""

    def __init__(self, seed: int):
        self.state = int(seed) & _MASK64

    def next_u64(self, n: int) -> np.ndarray:
        idx = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + idx * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        self.state = (self.state + n * int(_GOLDEN)) & _MASK64
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u


def derive_seed(seed: int, idx: int) -> int:
    """Per-instance seed: seed * 2^32 + idx (instances, samples)."""
    return (int(seed) * (1 << 32) + int(idx)) & _MASK64


# --------------------------------------------------------------------------
# 2-D shallow water
# --------------------------------------------------------------------------

@dataclass
class SWInput:
    """Interior-cell fields, row-major (ny, nx), x fastest, FP64."""
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    H: np.ndarray      # still-water depth (m); negative = land above datum
    eta0: np.ndarray   # initial surface elevation (m), already >= -H
    g: float = 9.81
    eps: float = 0.05
    hmin: float = 0.05

    def params(self) -> dict:
        return dict(nx=self.nx, ny=self.ny, dx=self.dx, dy=self.dy, dt=self.dt,
                    g=self.g, eps=self.eps, hmin=self.hmin)


def cell_centres(n: int, d: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * d


def sw_hump(n: int = 100, dx: float = 10.0, dt: float = 0.1, depth: float = 10.0,
            amp: float = 1.0, sigma_cells: float = 5.0) -> SWInput:
    """Flat basin with a Gaussian hump at the geometric centre (mirror symmetric)."""
    xc = cell_centres(n, dx)
    L = n * dx
    r2 = (xc[None, :] - L / 2) ** 2 + (xc[:, None] - L / 2) ** 2
    sig = sigma_cells * dx
    eta0 = amp * np.exp(-r2 / (2.0 * sig * sig))
    H = np.full((n, n), depth)
    return SWInput(n, n, dx, dx, dt, H, eta0)


def _gaussian_hills(nx, ny, centres_x, centres_y, sig, amp, xs=None, ys=None):
    """Sum of separable Gaussians evaluated at cell indices (xs, ys)."""
    xs = np.arange(nx, dtype=np.float64) + 0.5 if xs is None else xs
    ys = np.arange(ny, dtype=np.float64) + 0.5 if ys is None else ys
    out = np.zeros((ys.size, xs.size))
    for cx, cy, s in zip(centres_x, centres_y, sig):
        gx = np.exp(-((xs - cx) ** 2) / (2 * s * s))
        gy = np.exp(-((ys - cy) ** 2) / (2 * s * s))
        out += amp * np.outer(gy, gx)
    return out


def _surface_modes(nx, ny, rng: SplitMix64, nmodes=8, lmin=64.0, lmax=512.0):
    wl = np.exp(rng.uniform(nmodes, math.log(lmin), math.log(lmax)))
    ang = rng.uniform(nmodes, 0.0, 2 * math.pi)
    phi = rng.uniform(nmodes, 0.0, 2 * math.pi)
    return wl, ang, phi


def _eval_modes(wl, ang, phi, xs, ys):
    out = np.zeros((ys.size, xs.size))
    for w, a, p in zip(wl, ang, phi):
        kx = 2 * math.pi / w * math.cos(a)
        ky = 2 * math.pi / w * math.sin(a)
        # cos(kx x + ky y + p) = cos(kx x + p) cos(ky y) - sin(kx x + p) sin(ky y)
        out += np.outer(np.cos(ky * ys), np.cos(kx * xs + p)) - np.outer(np.sin(ky * ys), np.sin(kx * xs + p))
    return out


def sw_wetdry(n: int = 4096, seed: int = 1001, dx: float = 10.0, dt: float = 0.1,
              mean_depth: float = 50.0, hill_amp: float = 60.0, n_hills: int = 32,
              surf_amp: float = 0.5, dry_target: float = 0.15, hmin: float = 0.05,
              sample: int = 512, bisect_iters: int = 40) -> SWInput:
    """Random bathymetry with ~15 % dry land and a random-phase surface perturbation.

    H = mean_depth - sum_k hill_amp * exp(-|x - c_k|^2 / (2 sigma_k^2)), with
    sigma_k = s * U[0.5, 1.5]; the global width s is bisected on a sub-sampled
    copy of the grid so that the dry fraction (H + eta0 <= hmin) is
    dry_target, then re-checked at full resolution.
    """
    rng = SplitMix64(seed)
    cx = rng.uniform(n_hills, 0.0, n)
    cy = rng.uniform(n_hills, 0.0, n)
    sfac = rng.uniform(n_hills, 0.5, 1.5)
    wl, ang, phi = _surface_modes(n, n, rng, lmin=min(64.0, n / 4), lmax=min(512.0, n))

    stride = max(1, n // sample)
    xs = np.arange(0, n, stride, dtype=np.float64) + 0.5
    modes_s = _eval_modes(wl, ang, phi, xs, xs)
    eta_s = surf_amp * modes_s / np.abs(modes_s).max()

    def dry_frac(s, xs_, eta_):
        Hs = mean_depth - _gaussian_hills(n, n, cx, cy, s * sfac, hill_amp, xs_, xs_)
        return float(np.mean(Hs + eta_ <= hmin))

    lo, hi = 1.0, float(n)
    for _ in range(bisect_iters):
        mid = 0.5 * (lo + hi)
        if dry_frac(mid, xs, eta_s) < dry_target:
            lo = mid
        else:
            hi = mid
    s = 0.5 * (lo + hi)

    full = np.arange(n, dtype=np.float64) + 0.5
    H = mean_depth - _gaussian_hills(n, n, cx, cy, s * sfac, hill_amp, full, full)
    modes = _eval_modes(wl, ang, phi, full, full)
    eta_init = surf_amp * modes / np.abs(modes).max()
    eta0 = np.maximum(eta_init, -H)
    return SWInput(n, n, dx, dx, dt, H, eta0, hmin=hmin)


def sw_ensemble_sizes(count: int = 512, seed: int = 1002, nmin: int = 64, nmax: int = 1024) -> np.ndarray:
    """Square sides N = round(nmin * (nmax/nmin)^U), U ~ U[0, 1)."""
    rng = SplitMix64(seed)
    u = rng.uniform(count)
    return np.rint(nmin * (nmax / nmin) ** u).astype(np.int64)


def sw_ensemble_member(n: int, seed: int, idx: int, dx: float = 10.0, dt: float = 0.1) -> SWInput:
    """One ensemble instance: its own wet/dry bathymetry plus the 1 m, 5-cell hump."""
    base = sw_wetdry(n, derive_seed(seed, idx), dx=dx, dt=dt, sample=64, bisect_iters=24)
    xc = np.arange(n, dtype=np.float64) + 0.5
    r2 = (xc[None, :] - n / 2) ** 2 + (xc[:, None] - n / 2) ** 2
    hump = np.exp(-r2 / (2.0 * 25.0))
    eta0 = np.maximum(base.eta0 + hump, -base.H)
    return SWInput(n, n, dx, dx, dt, base.H, eta0)


# --------------------------------------------------------------------------
# Urban LES
# --------------------------------------------------------------------------

def les_buildings(nx: int, ny: int, nz: int, dx: float = 4.0, seed: int = 1003,
                  cover: float = 0.20, foot=(10.0, 40.0), height=(10.0, 60.0),
                  margin_cells: int | None = None) -> np.ndarray:
    """Solid mask (nz, ny, nx) uint8 of random rectangular blocks.

    Footprints U[foot] metres per side, heights U[height] metres, placed at
    uniform positions (kept ``margin_cells`` away from the inflow and outflow
    planes) until the union covers at least ``cover`` of the ground.
    """
    rng = SplitMix64(seed)
    if margin_cells is None:
        margin_cells = max(2, nx // 16)
    ground = np.zeros((ny, nx), dtype=bool)
    solid = np.zeros((nz, ny, nx), dtype=np.uint8)
    fmin = max(1, int(round(foot[0] / dx)))
    fmax = max(fmin, int(round(foot[1] / dx)))
    hmin_c = max(1, int(round(height[0] / dx)))
    hmax_c = max(hmin_c, int(round(height[1] / dx)))
    lo_x, hi_x = margin_cells, nx - margin_cells
    guard = 0
    while ground.mean() < cover and guard < 100000:
        guard += 1
        r = rng.uniform(5)
        wx = fmin + int(r[0] * (fmax - fmin + 1))
        wy = fmin + int(r[1] * (fmax - fmin + 1))
        hz = min(nz - 1, hmin_c + int(r[2] * (hmax_c - hmin_c + 1)))
        if hi_x - lo_x <= wx:
            break
        x0 = lo_x + int(r[3] * (hi_x - lo_x - wx))
        y0 = int(r[4] * ny)
        ys = np.arange(y0, y0 + wy) % ny
        ground[np.ix_(ys, np.arange(x0, x0 + wx))] = True
        solid[:hz][:, ys[:, None], np.arange(x0, x0 + wx)[None, :]] = 1
    return solid

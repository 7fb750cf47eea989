"""FP64 oracle of the learned warm start's grid transfers (test infrastructure).

Only tests, the smoke check and the benchmark's CPU leg use this module.

The pressure solve of the urban LES (Sec. 6.3.1 of arXiv:1711.04471) is
red-black SOR, whose iteration count is set by the smoothest error modes:
with Neumann walls at the inflow, ground and lid, periodic y and a Dirichlet
outflow, the slowest mode is a quarter cosine along x, constant over the
y-z planes.  A network that is to shorten the solve must therefore see the
whole domain, so the warm start runs it on a grid coarsened by a factor f in
each direction:

    r      = b - A p_prev                       (fine residual of the previous pressure)
    r_c    = prolong^T r / f^3                  (full-weighting restriction)
    p_c    = prolong^T p_prev / f^3
    s      = (f dx)^2 rms(r_c)                  (scale of the coarse increment)
    x      = [r_c / rms(r_c), p_c / rms(p_c)]   (network input, 2 channels)
    target = block mean of (p - p_prev) / s     (p the converged pressure)
    guess  = p_prev + s * prolong(out)          (out the network's output)

The input is restricted with the adjoint of the prolongation (the
restriction of Galerkin coarse-grid correction), which keeps the inner
product of r with every prolongated coarse field: the projection of r on the
slowest mode, which sets that mode's amplitude in p - p_prev, is kept to
second order, where block means lose the variation of the mode inside a
block.

prolong is trilinear interpolation between coarse cell centres: fine cell i
(0-based) sits at coarse coordinate (i + 1/2)/f - 1/2.  Beyond the end
centres it follows the boundary rules of the Poisson operator: the end value
is held at the inflow, the ground and the lid (Neumann: mirror ghost), the
ghost past the outflow is minus the last value (p = 0 on the outflow face),
and y wraps around (periodic).
"""
from __future__ import annotations

import math

import numpy as np

from . import les as ol


def restrict(a: np.ndarray, f: int) -> np.ndarray:
    """Block mean of a (nz, ny, nx) array over f x f x f blocks."""
    nz, ny, nx = a.shape
    if nz % f or ny % f or nx % f:
        raise ValueError("grid not divisible by f")
    return a.reshape(nz // f, f, ny // f, f, nx // f, f).mean(axis=(1, 3, 5))


def _axis_weights(n: int, nc: int, f: int, rule: str) -> np.ndarray:
    """(n, nc) matrix of linear-interpolation weights along one axis; rule is
    "periodic", "neumann" (both ends held) or "outflow" (held at the first
    end, antisymmetric ghost past the last)."""
    M = np.zeros((n, nc))
    for i in range(n):
        X = (i + 0.5) / f - 0.5
        if rule == "periodic":
            i0 = math.floor(X)
            w = X - i0
            M[i, i0 % nc] += 1.0 - w
            M[i, (i0 + 1) % nc] += w
            continue
        X = max(X, 0.0)
        if rule == "neumann":
            X = min(X, nc - 1.0)
        i0 = min(int(math.floor(X)), nc - 1)
        w = X - i0
        M[i, i0] += 1.0 - w
        if i0 + 1 < nc:
            M[i, i0 + 1] += w
        elif rule == "outflow":
            M[i, nc - 1] -= w     # ghost = -last value
    return M


def _weights(nz: int, ny: int, nx: int, f: int):
    return (_axis_weights(nz, nz // f, f, "neumann"), _axis_weights(ny, ny // f, f, "periodic"),
            _axis_weights(nx, nx // f, f, "outflow"))


def prolong(c: np.ndarray, f: int) -> np.ndarray:
    """Trilinear interpolation of a coarse (ncz, ncy, ncx) field to the fine grid."""
    ncz, ncy, ncx = c.shape
    Wz, Wy, Wx = _weights(ncz * f, ncy * f, ncx * f, f)
    # one axis at a time (a sequence of matrix products), not one 6-index loop
    return np.einsum("zk,yj,xi,kji->zyx", Wz, Wy, Wx, c, optimize=True)


def restrict_fw(a: np.ndarray, f: int) -> np.ndarray:
    """Full weighting: prolong^T a / f^3 for a fine (nz, ny, nx) field."""
    nz, ny, nx = a.shape
    if nz % f or ny % f or nx % f:
        raise ValueError("grid not divisible by f")
    Wz, Wy, Wx = _weights(nz, ny, nx, f)
    return np.einsum("zk,yj,xi,zyx->kji", Wz, Wy, Wx, a, optimize=True) / f ** 3


def residual_field(P, b: np.ndarray, p: np.ndarray) -> np.ndarray:
    """Interior r = b - A p from padded b, p (the LES oracle's operator)."""
    return ol.interior(b) - ol.interior(ol.apply_A(P, np.ascontiguousarray(p, dtype=np.float64)))


def features(P, b: np.ndarray, p_prev: np.ndarray, f: int):
    """Network input (ncz, ncy, ncx, 2) and scale s from padded b and p_prev."""
    r = residual_field(P, np.ascontiguousarray(b, dtype=np.float64), p_prev)
    rc = restrict_fw(r, f)
    pc = restrict_fw(np.asarray(ol.interior(p_prev), dtype=np.float64), f)
    rms_r = math.sqrt(float(np.mean(rc * rc)))
    rms_p = math.sqrt(float(np.mean(pc * pc)))
    x = np.stack([rc / rms_r if rms_r > 0 else np.zeros_like(rc), pc / rms_p if rms_p > 0 else np.zeros_like(pc)],
                 axis=-1)
    return x, (f * P.dx) ** 2 * rms_r


def target(p_prev: np.ndarray, p_new: np.ndarray, f: int, s: float) -> np.ndarray:
    """Coarse training target from padded p_prev and the converged p_new."""
    return restrict(ol.interior(p_new) - ol.interior(p_prev), f) / s


def apply(p_prev: np.ndarray, out: np.ndarray, s: float, f: int) -> np.ndarray:
    """Padded warm start p_prev + s * prolong(out); the halo is copied."""
    p = np.array(p_prev, dtype=np.float64)
    p[1:-1, 1:-1, 1:-1] += s * prolong(np.asarray(out, dtype=np.float64), f)
    return p

"""Pins of the FP64 UFLES oracle against mathematics and the stated setup.

Each test checks a property fixed independently of the oracle's code: a
dense direct solve, the continuum solution, exactness of second-order
central differences on polynomial fields, the order of Adams-Bashforth,
the discrete divergence theorem after projection, and the stated inflow
profile (5 m/s at 10 m).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import les

oracle.lib()


# ---------------------------------------------------------------- Poisson

def _dense_A(nx, ny, nz, dx):
    """Assemble the pressure operator from the boundary rules, cell by cell:
    mirror ghost (Neumann) at x=0, z=0, z=top; antisymmetric ghost (p = 0 on
    the face, Dirichlet) at x=L; periodic in y."""
    n = nx * ny * nz
    idx = lambda i, j, k: (k * ny + j) * nx + i
    A = np.zeros((n, n))
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = idx(i, j, k)
                for di, dj, dk in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    A[r, r] -= 1.0
                    ii, jj, kk = i + di, (j + dj) % ny, k + dk
                    if ii < 0 or kk < 0 or kk >= nz:        # mirror ghost equals the cell itself
                        A[r, r] += 1.0
                    elif ii >= nx:                           # ghost = -cell
                        A[r, r] -= 1.0
                    else:
                        A[r, idx(ii, jj, kk)] += 1.0
    return A / dx ** 2


def test_poisson_sor_matches_dense_solve():
    nx, ny, nz, dx = 8, 6, 7, 4.0
    P = les.make_params(nx, ny, nz, dx=dx)
    rng = np.random.default_rng(1)
    b_int = rng.standard_normal((nz, ny, nx))
    x = np.linalg.solve(_dense_A(nx, ny, nz, dx), b_int.ravel()).reshape(nz, ny, nx)
    b = les.padded(P)
    les.interior(b)[:] = b_int
    p = les.padded(P)
    rc, it, rr = les.sor(P, b, p, omega=1.8, tol=1e-13, max_iter=200000)
    assert rc == 0 and rr <= 1e-13
    assert np.abs(les.interior(p) - x).max() <= 1e-10 * np.abs(x).max()


def test_poisson_second_order_against_continuum():
    """p = cos(pi x / 2L) cos(2 pi y / L) cos(pi z / L) meets every boundary
    rule; the discrete solution converges to it at second order."""
    errs = []
    for n in (8, 16, 32):
        L = 1.0
        dx = L / n
        P = les.make_params(n, n, n, dx=dx)
        c = (np.arange(n) + 0.5) * dx
        Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
        kx, ky, kz = math.pi / (2 * L), 2 * math.pi / L, math.pi / L
        pe = np.cos(kx * X) * np.cos(ky * Y) * np.cos(kz * Z)
        b = les.padded(P)
        les.interior(b)[:] = -(kx ** 2 + ky ** 2 + kz ** 2) * pe
        p = les.padded(P)
        rc, it, rr = les.sor(P, b, p, omega=1.9, tol=1e-11, max_iter=500000)
        assert rc == 0
        errs.append(np.abs(les.interior(p) - pe).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5, errs


def test_residual_is_relative_to_b():
    P = les.make_params(6, 6, 6)
    b = les.padded(P)
    les.interior(b)[:] = 1.0
    p = les.padded(P)
    assert abs(les.residual(P, b, p) - 1.0) < 1e-15
    assert les.sor(P, les.padded(P), p)[1] == 0   # b = 0: converged with no iteration


# ------------------------------------------------------ polynomial fields

def _positions(P):
    """Coordinates (padded index space) of u, v, w faces and cell centres."""
    d = P.dx
    i = np.arange(P.nx + 2)
    j = np.arange(P.ny + 2)
    k = np.arange(P.nz + 2)
    K, J, I = np.meshgrid(k, j, i, indexing="ij")
    xc, yc, zc = (I - 0.5) * d, (J - 0.5) * d, (K - 0.5) * d
    return dict(u=(I * d, yc, zc), v=(xc, J * d, zc), w=(xc, yc, K * d), c=(xc, yc, zc))


def _linear_fields(P, seed=0):
    rng = np.random.default_rng(seed)
    a, b, c = rng.standard_normal(4), rng.standard_normal(4), rng.standard_normal(4)
    pos = _positions(P)
    f = lambda co, x: co[0] + co[1] * x[0] + co[2] * x[1] + co[3] * x[2]
    return a, b, c, f(a, pos["u"]), f(b, pos["v"]), f(c, pos["w"]), pos


def test_velfg_exact_for_linear_velocity():
    P = les.make_params(7, 6, 5, dx=0.5)
    a, b, c, u, v, w, pos = _linear_fields(P)
    fu, fv, fw = les.velfg(P, u, v, w)
    ev = lambda co, x: co[0] + co[1] * x[0] + co[2] * x[1] + co[3] * x[2]
    # -div(u (x) u) at each face for u = a.x, v = b.x, w = c.x (gradients a[1:], b[1:], c[1:])
    U, V, W = (ev(a, pos["u"]), ev(b, pos["u"]), ev(c, pos["u"]))
    cu = 2 * U * a[1] + a[2] * V + U * b[2] + a[3] * W + U * c[3]
    U, V, W = (ev(a, pos["v"]), ev(b, pos["v"]), ev(c, pos["v"]))
    cv = b[1] * U + V * a[1] + 2 * V * b[2] + b[3] * W + V * c[3]
    U, V, W = (ev(a, pos["w"]), ev(b, pos["w"]), ev(c, pos["w"]))
    cw = c[1] * U + W * a[1] + c[2] * V + W * b[2] + 2 * W * c[3]
    sl = (slice(1, -1), slice(1, -1), slice(1, -1))
    slw = (slice(1, -2), slice(1, -1), slice(1, -1))
    scale = max(np.abs(cu).max(), 1.0)
    assert np.abs(fu[sl] + cu[sl]).max() <= 1e-12 * scale
    assert np.abs(fv[sl] + cv[sl]).max() <= 1e-12 * scale
    assert np.abs(fw[slw] + cw[slw]).max() <= 1e-12 * scale
    assert np.all(fw[-2, 1:-1, 1:-1] == 0.0)


def test_viscous_term_exact_for_quadratic_velocity():
    """With nu_t = 0 and constant nu, div(2 nu S) = nu (lap u + grad div u)
    holds exactly for quadratic fields."""
    P = les.make_params(6, 7, 5, dx=0.5, cs=0.0, nu=0.3)
    pos = _positions(P)
    rng = np.random.default_rng(2)
    Q = rng.standard_normal((3, 10))  # coefficients of 1, x, y, z, x2, y2, z2, xy, xz, yz

    def field(q, x):
        X, Y, Z = x
        return q[0] + q[1] * X + q[2] * Y + q[3] * Z + q[4] * X * X + q[5] * Y * Y + q[6] * Z * Z + \
            q[7] * X * Y + q[8] * X * Z + q[9] * Y * Z

    u, v, w = field(Q[0], pos["u"]), field(Q[1], pos["v"]), field(Q[2], pos["w"])
    fu, fv, fw = les.padded(P), les.padded(P), les.padded(P)
    les.visc(P, u, v, w, les.padded(P), fu, fv, fw)
    lap = lambda q: 2 * (q[4] + q[5] + q[6])
    # grad(div u): div = (q1+2q4 x+q7 y+q8 z)_u + (q2+q7 x+2q5 y+q9 z)_v + (q3+q8 x+q9 y+2q6 z)_w
    gdiv = np.array([2 * Q[0][4] + Q[1][7] + Q[2][8], Q[0][7] + 2 * Q[1][5] + Q[2][9], Q[0][8] + Q[1][9] + 2 * Q[2][6]])
    nu = 0.3
    sl = (slice(1, -1), slice(1, -1), slice(1, -1))
    slw = (slice(1, -2), slice(1, -1), slice(1, -1))
    assert np.abs(fu[sl] - nu * (lap(Q[0]) + gdiv[0])).max() <= 1e-11
    assert np.abs(fv[sl] - nu * (lap(Q[1]) + gdiv[1])).max() <= 1e-11
    assert np.abs(fw[slw] - nu * (lap(Q[2]) + gdiv[2])).max() <= 1e-11


def test_smagorinsky_viscosity_for_uniform_strain():
    P = les.make_params(6, 5, 4, dx=0.5, cs=0.1)
    a, b, c, u, v, w, pos = _linear_fields(P, seed=4)
    G = np.array([a[1:], b[1:], c[1:]])        # G[i][j] = d u_i / d x_j
    S = 0.5 * (G + G.T)
    expect = (0.1 * 0.5) ** 2 * math.sqrt(2.0 * np.sum(S * S))
    nt = les.nut(P, u, v, w)
    assert np.abs(les.interior(nt) - expect).max() <= 1e-13
    assert np.array_equal(nt[0, 1:-1, 1:-1], nt[1, 1:-1, 1:-1])    # zero gradient at the ground


def test_adams_bashforth_is_second_order():
    lam, T = -0.7, 2.0
    errs = []
    for nsteps in (40, 80, 160):
        P = les.make_params(3, 2, 2, dt=T / nsteps)
        u, v, w = les.padded(P), les.padded(P), les.padded(P)
        fuo, fvo, fwo = les.padded(P), les.padded(P), les.padded(P)
        u[1:-1, 1:-1, 1:-1] = 1.0
        for s in range(nsteps):
            fu, fv, fw = lam * u, lam * v, lam * w
            les.adam(P, s == 0, u, v, w, fu, fv, fw, fuo, fvo, fwo)
        errs.append(abs(u[1, 1, 1] - math.exp(lam * T)))
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4, errs


# ------------------------------------------------------------- full step

def _small_case():
    nx, ny, nz = 16, 12, 10
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:4, 3:6, 5:8] = 1
    solid[:2, 8:11, 9:12] = 1
    return les.make_params(nx, ny, nz), solid


def test_projection_matches_poisson_residual():
    """After velnw, div(u)/dt equals b - A p cell by cell (discrete divergence
    theorem with the same boundary rules), so the projected field is
    divergence-free to the solver tolerance."""
    P, solid = _small_case()
    s = les.LESState(P, solid).step(2)
    u, v, w = s.u.copy(), s.v.copy(), s.w.copy()
    b = les.rhs(P, u, v, w)
    r = b - les.apply_A(P, s.p)
    les.velnw(P, s.p, u, v, w)
    les.bondv1(P, u, v, w)
    div = les.rhs(P, u, v, w)
    assert np.abs(les.interior(div - r)).max() <= 1e-9 * np.abs(les.interior(b)).max()
    assert np.linalg.norm(les.interior(div)) <= 1.01e-6 * np.linalg.norm(les.interior(b))
    # net inflow through x = 0 equals net outflow through x = L
    qin = u[1:-1, 1:-1, 0].sum()
    qout = u[1:-1, 1:-1, P.nx].sum()
    assert abs(qin - qout) <= 1e-6 * abs(qin) * P.nx * P.ny * P.nz


def test_inflow_profile_is_5_m_per_s_at_10_m():
    P = les.make_params(4, 4, 6, dx=4.0)
    u, v, w = les.padded(P), les.padded(P), les.padded(P)
    les.bondv1(P, u, v, w)
    assert abs(u[3, 2, 0] - 5.0) < 1e-12           # face centre height (3 - 1/2) * 4 = 10 m
    assert u[1, 2, 0] < u[2, 2, 0] < u[3, 2, 0] < u[6, 2, 0]


def test_bondv1_wall_rules():
    P = les.make_params(5, 4, 6)
    rng = np.random.default_rng(3)
    u, v, w = (rng.standard_normal((P.nz + 2, P.ny + 2, P.nx + 2)) for _ in range(3))
    les.bondv1(P, u, v, w)
    assert np.allclose(u[0] + u[1], 0) and np.allclose(v[0] + v[1], 0)     # no slip at the ground
    assert np.array_equal(u[-1], u[-2]) and np.array_equal(v[-1], v[-2])   # free slip at the lid
    assert not w[0].any() and not w[P.nz].any()
    assert np.array_equal(u[1:-1, 0, :], u[1:-1, P.ny, :])                  # periodic in y


def test_goldstein_forcing_stops_flow_in_buildings():
    P, solid = _small_case()
    s = les.LESState(P, solid).step(200)
    S = solid.astype(bool)
    inside_u = S & np.concatenate([S[:, :, 1:], np.ones_like(S[:, :, :1])], axis=2)   # both cells solid
    umax = np.abs(s.u[1:-1, 1:-1, 1:-1][inside_u]).max()
    assert umax < 1e-2 * 5.0, umax
    assert all(h[2] == 0 for h in s.history)                # every solve converged
    assert np.abs(s.u).max() < 20.0


def test_free_stream_without_buildings_keeps_log_profile_shape():
    """No buildings: the flow stays a shear flow driven by the inflow; w
    remains small compared with u and nothing blows up in 50 steps."""
    P = les.make_params(12, 8, 8)
    s = les.LESState(P, np.zeros((8, 8, 12), np.uint8)).step(50)
    um = les.interior(s.u).mean(axis=(1, 2))
    assert np.all(np.diff(um) > 0)                          # speed increases with height
    assert np.abs(s.w).max() < 0.2 * np.abs(s.u).max()

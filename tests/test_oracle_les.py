"""Pins of the FP64 UFLES oracle against mathematics and the stated setup.

Each test checks a property fixed independently of the oracle's code: a
dense direct solve, the continuum solution, exactness of second-order
central differences on polynomial fields (including the edge averages of
the Smagorinsky model, for a linear eddy viscosity and for the variance
term of a linear strain), the order of Adams-Bashforth, the discrete
divergence theorem after projection, the stated inflow profile (5 m/s at
10 m), and a position-keyed brute-force restatement of nu_t, the viscous
stress divergence and the Goldstein feedback on a 4 x 4 x 4 grid.
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


# ------------------------------------------- les / feedbf: closed forms
# Eq. (les) of Sec. 6.3.1 ("les: viscosity, Smagorinsky model") in this
# project's reading: nu_t = (cs dx)^2 sqrt(2 S:S) at cell centres, with the
# off-diagonal S_ij^2 averaged from the four edges around the centre, and
# F += div(2 (nu + nu_t) S) with nu_eff averaged from the four centres
# around each edge.  The fields below make every difference quotient exact,
# so the expected values follow from calculus alone.

_Q_NAMES = ("1", "x", "y", "z", "xx", "yy", "zz", "xy", "xz", "yz")


def _quad(q, pos):
    X, Y, Z = pos
    return q[0] + q[1] * X + q[2] * Y + q[3] * Z + q[4] * X * X + q[5] * Y * Y + q[6] * Z * Z + \
        q[7] * X * Y + q[8] * X * Z + q[9] * Y * Z


def _quad_grad(q, pos):
    """Gradient (d/dx, d/dy, d/dz) of the quadratic with coefficients q."""
    X, Y, Z = pos
    return (q[1] + 2 * q[4] * X + q[7] * Y + q[8] * Z,
            q[2] + 2 * q[5] * Y + q[7] * X + q[9] * Z,
            q[3] + 2 * q[6] * Z + q[8] * X + q[9] * Y)


def _strain(Q, pos):
    """S_ij = (du_i/dx_j + du_j/dx_i) / 2 of the quadratic velocity Q at pos."""
    G = [_quad_grad(Q[a], pos) for a in range(3)]       # G[a][b] = d u_a / d x_b
    return [[0.5 * (G[a][b] + G[b][a]) for b in range(3)] for a in range(3)]


def test_smagorinsky_edge_average_of_quadratic_velocity():
    """For a quadratic velocity the strain S is linear.  The centred
    differences give S_11, S_22, S_33 at the centre and S_12, S_13, S_23 at
    the edges exactly, so the mean of S_12^2 over the four edges around a
    centre is S_12(c)^2 + h^2 (|dS_12/dx|^2 + |dS_12/dy|^2) with h = dx/2
    (the cross terms cancel by symmetry).  A shifted or dropped edge changes
    that value."""
    P = les.make_params(5, 6, 4, dx=0.5, cs=0.1)
    pos = _positions(P)
    rng = np.random.default_rng(11)
    Q = rng.standard_normal((3, 10))
    u, v, w = _quad(Q[0], pos["u"]), _quad(Q[1], pos["v"]), _quad(Q[2], pos["w"])
    nt = les.nut(P, u, v, w)
    h = 0.5 * P.dx
    # gradient of the (linear) S_ij: d S_ij / d x_b = (d2u_i/dx_j dx_b + d2u_j/dx_i dx_b) / 2
    H = np.zeros((3, 3, 3))                 # H[a][j][b] = d2 u_a / dx_j dx_b
    for a in range(3):
        q = Q[a]
        H[a] = [[2 * q[4], q[7], q[8]], [q[7], 2 * q[5], q[9]], [q[8], q[9], 2 * q[6]]]
    dS = 0.5 * (H + H.transpose(1, 0, 2))   # dS[i][j][b]
    worst = 0.0
    for k in range(1, P.nz + 1):
        for j in range(1, P.ny + 1):
            for i in range(1, P.nx + 1):
                c = tuple(p[k, j, i] for p in pos["c"])
                S = _strain(Q, c)
                ss = 2 * (S[0][0] ** 2 + S[1][1] ** 2 + S[2][2] ** 2)
                for (a, b) in ((0, 1), (0, 2), (1, 2)):
                    mean_sq = S[a][b] ** 2 + h * h * (dS[a][b][a] ** 2 + dS[a][b][b] ** 2)
                    ss += 4 * mean_sq
                expect = (P.cs * P.dx) ** 2 * math.sqrt(ss)
                worst = max(worst, abs(nt[k, j, i] - expect) / expect)
    assert worst <= 1e-13, worst


def test_viscous_term_exact_for_linear_eddy_viscosity():
    """Quadratic velocity and nu_eff = nu + nu_t linear in space (nu_t given
    at every centre, ghosts included): the centre and edge values of
    2 nu_eff S are exact point values of a quadratic, so the flux-difference
    divergence is the exact d/dx_j (2 nu_eff S_ij) at each face,
    2 grad(nu_eff) . S_i + nu_eff (lap u_i + d/dx_i div u).  The four-centre
    average of nu_eff is exact at the edge only if the four centres are the
    right ones."""
    P = les.make_params(6, 5, 5, dx=0.5, cs=0.1, nu=0.2)
    pos = _positions(P)
    rng = np.random.default_rng(12)
    Q = rng.standard_normal((3, 10))
    g_nu = rng.standard_normal(3) * 0.3
    nu0 = 3.0
    nut_field = nu0 - P.nu + g_nu[0] * pos["c"][0] + g_nu[1] * pos["c"][1] + g_nu[2] * pos["c"][2]
    u, v, w = _quad(Q[0], pos["u"]), _quad(Q[1], pos["v"]), _quad(Q[2], pos["w"])
    fu, fv, fw = les.padded(P), les.padded(P), les.padded(P)
    les.visc(P, u, v, w, np.ascontiguousarray(nut_field), fu, fv, fw)

    def expect(a, x):
        S = _strain(Q, x)
        X, Y, Z = x
        nu_e = nu0 + g_nu[0] * X + g_nu[1] * Y + g_nu[2] * Z
        q = Q[a]
        lap = 2 * (q[4] + q[5] + q[6])
        # d/dx_a of div u
        gd = [2 * Q[0][4] + Q[1][7] + Q[2][8], Q[0][7] + 2 * Q[1][5] + Q[2][9], Q[0][8] + Q[1][9] + 2 * Q[2][6]]
        return 2 * sum(g_nu[b] * S[a][b] for b in range(3)) + nu_e * (lap + gd[a])

    worst = 0.0
    for a, (f, key) in enumerate(((fu, "u"), (fv, "v"), (fw, "w"))):
        kmax = P.nz - 1 if a == 2 else P.nz
        for k in range(1, kmax + 1):
            for j in range(1, P.ny + 1):
                for i in range(1, P.nx + 1):
                    e = expect(a, tuple(p[k, j, i] for p in pos[key]))
                    worst = max(worst, abs(f[k, j, i] - e) / (1.0 + abs(e)))
    assert worst <= 1e-12, worst


def test_goldstein_integral_includes_the_current_velocity():
    """feedbf on faces that touch a building: the time integral is advanced
    first, G <- G + dt u, and the force uses the advanced integral,
    F <- F + alpha G + beta u (reading of the Goldstein feedback of Sec.
    6.3.1; the rectangle rule at the right end of the step).  Faces that
    touch no building, the lid w faces and every ghost are unchanged."""
    nx, ny, nz = 5, 4, 4
    P = les.make_params(nx, ny, nz, dt=0.05, alpha=-7.0, beta=-3.0)
    rng = np.random.default_rng(13)
    shp = (nz + 2, ny + 2, nx + 2)
    u, v, w, gu, gv, gw, fu, fv, fw = (rng.standard_normal(shp) for _ in range(9))
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[0, 1, 2] = 1          # cell (i, j, k) = (3, 2, 1)
    solid[3, 3, 4] = 1          # (5, 4, 4): the outflow column, the last y row and the lid layer
    G0 = [a.copy() for a in (gu, gv, gw)]
    F0 = [a.copy() for a in (fu, fv, fw)]
    les.feedbf(P, solid, u, v, w, gu, gv, gw, fu, fv, fw)
    S = lambda i, j, k: 1 <= i <= nx and 1 <= k <= nz and bool(solid[k - 1, (j - 1) % ny, i - 1])
    for a, (vel, g, f) in enumerate(((u, gu, fu), (v, gv, fv), (w, gw, fw))):
        for k in range(nz + 2):
            for j in range(ny + 2):
                for i in range(nx + 2):
                    inside = 1 <= i <= nx and 1 <= j <= ny and 1 <= k <= (nz - 1 if a == 2 else nz)
                    nb = [(i, j, k), (i + 1, j, k) if a == 0 else (i, j + 1, k) if a == 1 else (i, j, k + 1)]
                    touched = inside and any(S(*c) for c in nb)
                    if touched:
                        g_new = G0[a][k, j, i] + P.dt * vel[k, j, i]
                        f_new = F0[a][k, j, i] + P.alpha * g_new + P.beta * vel[k, j, i]
                        assert abs(g[k, j, i] - g_new) <= 1e-15 * (1 + abs(g_new))
                        assert abs(f[k, j, i] - f_new) <= 1e-14 * (1 + abs(f_new)), (a, i, j, k)
                    else:
                        assert g[k, j, i] == G0[a][k, j, i] and f[k, j, i] == F0[a][k, j, i], (a, i, j, k)
    # the building at (3, 2, 1) forces both u faces of its cell
    assert fu[1, 2, 2] != F0[0][1, 2, 2] and fu[1, 2, 3] != F0[0][1, 2, 3]
    # the lid w face of (5, 4, 4) is not forced; the y wrap forces v of (5, 4, 4) and v of (5, 0 -> 4, 4)
    assert fw[4, 4, 5] == F0[2][4, 4, 5] and fv[4, 4, 5] != F0[1][4, 4, 5]


# ------------------------------------ les / feedbf: brute-force transcription
# An independent restatement of the same formulas on a 4 x 4 x 4 grid: fields
# are dictionaries keyed by the position of each value in half-cell units
# (cell centres at odd coordinates, faces and edges at even ones), and every
# stencil is written as offsets of those positions, with no array indexing.

def _to_dict(a, kind):
    """Padded array -> {(X, Y, Z): value} in half-cell units."""
    off = {"c": (-1, -1, -1), "u": (0, -1, -1), "v": (-1, 0, -1), "w": (-1, -1, 0)}[kind]
    d = {}
    for k in range(a.shape[0]):
        for j in range(a.shape[1]):
            for i in range(a.shape[2]):
                d[(2 * i + off[0], 2 * j + off[1], 2 * k + off[2])] = float(a[k, j, i])
    return d


def _brute_nut(P, U, V, W):
    dx, l2 = P.dx, (P.cs * P.dx) ** 2
    centres = [(2 * i - 1, 2 * j - 1, 2 * k - 1) for k in range(1, P.nz + 1) for j in range(1, P.ny + 1)
               for i in range(1, P.nx + 1)]

    def s12(X, Y, Z):            # edge at even X, even Y
        return 0.5 * ((U[(X, Y + 1, Z)] - U[(X, Y - 1, Z)]) + (V[(X + 1, Y, Z)] - V[(X - 1, Y, Z)])) / dx

    def s13(X, Y, Z):            # edge at even X, even Z
        return 0.5 * ((U[(X, Y, Z + 1)] - U[(X, Y, Z - 1)]) + (W[(X + 1, Y, Z)] - W[(X - 1, Y, Z)])) / dx

    def s23(X, Y, Z):            # edge at even Y, even Z
        return 0.5 * ((V[(X, Y, Z + 1)] - V[(X, Y, Z - 1)]) + (W[(X, Y + 1, Z)] - W[(X, Y - 1, Z)])) / dx

    out = {}
    for (X, Y, Z) in centres:
        d11 = (U[(X + 1, Y, Z)] - U[(X - 1, Y, Z)]) / dx
        d22 = (V[(X, Y + 1, Z)] - V[(X, Y - 1, Z)]) / dx
        d33 = (W[(X, Y, Z + 1)] - W[(X, Y, Z - 1)]) / dx
        e12 = sum(s12(X + a, Y + b, Z) ** 2 for a in (-1, 1) for b in (-1, 1)) / 4
        e13 = sum(s13(X + a, Y, Z + b) ** 2 for a in (-1, 1) for b in (-1, 1)) / 4
        e23 = sum(s23(X, Y + a, Z + b) ** 2 for a in (-1, 1) for b in (-1, 1)) / 4
        out[(X, Y, Z)] = l2 * math.sqrt(2 * (d11 * d11 + d22 * d22 + d33 * d33) + 4 * (e12 + e13 + e23))
    # ghost centres: copy the nearest interior centre in x and z, wrap in y
    full = dict(out)
    for X in range(-1, 2 * P.nx + 2, 2):
        for Y in range(-1, 2 * P.ny + 2, 2):
            for Z in range(-1, 2 * P.nz + 2, 2):
                if (X, Y, Z) in full:
                    continue
                Xs = min(max(X, 1), 2 * P.nx - 1)
                Zs = min(max(Z, 1), 2 * P.nz - 1)
                Ys = (Y - 1) % (2 * P.ny) + 1
                full[(X, Y, Z)] = out[(Xs, Ys, Zs)]
    return full


def _brute_visc(P, U, V, W, NT):
    dx, nu = P.dx, P.nu
    ne = lambda c: nu + NT[c]

    def nu_edge(X, Y, Z, axes):
        pts = []
        for a in (-1, 1):
            for b in (-1, 1):
                p = [X, Y, Z]
                p[axes[0]] += a
                p[axes[1]] += b
                pts.append(tuple(p))
        return sum(ne(p) for p in pts) / 4

    def t_diag(X, Y, Z, a):       # at a centre
        F = (U, V, W)[a]
        e = [0, 0, 0]
        e[a] = 1
        hi = (X + e[0], Y + e[1], Z + e[2])
        lo = (X - e[0], Y - e[1], Z - e[2])
        return 2 * ne((X, Y, Z)) * (F[hi] - F[lo]) / dx

    def t_off(X, Y, Z, a, b):     # at the edge (even coordinates along a and b)
        Fa, Fb = (U, V, W)[a], (U, V, W)[b]
        ea = [0, 0, 0]
        eb = [0, 0, 0]
        ea[a] = 1
        eb[b] = 1
        pb = lambda s: (X + s * eb[0], Y + s * eb[1], Z + s * eb[2])
        pa = lambda s: (X + s * ea[0], Y + s * ea[1], Z + s * ea[2])
        s = 0.5 * ((Fa[pb(1)] - Fa[pb(-1)]) + (Fb[pa(1)] - Fb[pa(-1)])) / dx
        return 2 * nu_edge(X, Y, Z, (a, b)) * s

    res = []
    for a in range(3):
        faces = {}
        kmax = P.nz - 1 if a == 2 else P.nz
        for k in range(1, kmax + 1):
            for j in range(1, P.ny + 1):
                for i in range(1, P.nx + 1):
                    X, Y, Z = 2 * i - 1, 2 * j - 1, 2 * k - 1
                    if a == 0:
                        X += 1
                    elif a == 1:
                        Y += 1
                    else:
                        Z += 1
                    tot = 0.0
                    for b in range(3):
                        e = [0, 0, 0]
                        e[b] = 1
                        hi = (X + e[0], Y + e[1], Z + e[2])
                        lo = (X - e[0], Y - e[1], Z - e[2])
                        if b == a:
                            tot += t_diag(*hi, a) - t_diag(*lo, a)
                        else:
                            lo_ax, hi_ax = min(a, b), max(a, b)
                            tot += t_off(*hi, lo_ax, hi_ax) - t_off(*lo, lo_ax, hi_ax)
                    faces[(X, Y, Z)] = tot / dx
        res.append(faces)
    return res


def _brute_feedbf(P, solid, vel, G, F):
    nx, ny, nz = P.nx, P.ny, P.nz
    cell_solid = {}
    for k in range(1, nz + 1):
        for j in range(1, ny + 1):
            for i in range(1, nx + 1):
                cell_solid[(2 * i - 1, 2 * j - 1, 2 * k - 1)] = bool(solid[k - 1, j - 1, i - 1])

    def is_solid(X, Y, Z):
        Y = (Y - 1) % (2 * ny) + 1                  # periodic in y
        return cell_solid.get((X, Y, Z), False)     # outside x or z: no building

    for a in range(3):
        kmax = nz - 1 if a == 2 else nz
        for k in range(1, kmax + 1):
            for j in range(1, ny + 1):
                for i in range(1, nx + 1):
                    p = [2 * i - 1, 2 * j - 1, 2 * k - 1]
                    p[a] += 1
                    lo, hi = list(p), list(p)
                    lo[a] -= 1
                    hi[a] += 1
                    if is_solid(*lo) or is_solid(*hi):
                        key = tuple(p)
                        G[a][key] = G[a][key] + P.dt * vel[a][key]
                        F[a][key] = F[a][key] + P.alpha * G[a][key] + P.beta * vel[a][key]


def _compare(d, a, kind):
    """Largest relative difference between dictionary d and padded array a
    over the positions d holds."""
    ref = _to_dict(a, kind)
    scale = max(abs(x) for x in d.values()) + 1e-300
    return max(abs(ref[k] - val) for k, val in d.items()) / scale


def test_brute_force_les_4x4x4():
    """nut, the viscous stress divergence (with a random non-zero nu_t) and
    feedbf against the position-keyed transcription, to 1e-13."""
    P = les.make_params(4, 4, 4, dx=2.0, cs=0.17, nu=0.05, dt=0.03, alpha=-50.0, beta=-4.0)
    rng = np.random.default_rng(14)
    shp = (P.nz + 2, P.ny + 2, P.nx + 2)
    u, v, w = (rng.standard_normal(shp) for _ in range(3))
    U, V, W = _to_dict(u, "u"), _to_dict(v, "v"), _to_dict(w, "w")

    # nut (interior and ghost centres)
    nt = les.nut(P, u, v, w)
    NT = _brute_nut(P, U, V, W)
    assert _compare(NT, nt, "c") <= 1e-13

    # viscous term with an unrelated, strictly positive nu_t on every centre
    nt_rand = np.ascontiguousarray(rng.uniform(0.1, 2.0, shp))
    fu, fv, fw = les.padded(P), les.padded(P), les.padded(P)
    les.visc(P, u, v, w, nt_rand, fu, fv, fw)
    BU, BV, BW = _brute_visc(P, U, V, W, _to_dict(nt_rand, "c"))
    assert _compare(BU, fu, "u") <= 1e-13
    assert _compare(BV, fv, "v") <= 1e-13
    assert _compare(BW, fw, "w") <= 1e-13

    # feedbf with buildings on the x and y edges of the grid and the lid
    solid = (rng.random((P.nz, P.ny, P.nx)) < 0.3).astype(np.uint8)
    solid[3, 3, 3] = 1
    gs = [rng.standard_normal(shp) for _ in range(3)]
    fs = [rng.standard_normal(shp) for _ in range(3)]
    G = [_to_dict(g, k) for g, k in zip(gs, "uvw")]
    F = [_to_dict(f, k) for f, k in zip(fs, "uvw")]
    les.feedbf(P, solid, u, v, w, *gs, *fs)
    _brute_feedbf(P, solid, (U, V, W), G, F)
    for a, kind in enumerate("uvw"):
        ref_g, ref_f = _to_dict(gs[a], kind), _to_dict(fs[a], kind)
        assert max(abs(ref_g[k] - G[a][k]) for k in G[a]) <= 1e-13
        assert max(abs(ref_f[k] - F[a][k]) for k in F[a]) <= 1e-13

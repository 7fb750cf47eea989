"""Parity of the CUDA UFLES step and pressure solve (through the C ABI)
with the FP64 oracle.

FP32 fields: relative L2 error <= 1e-5 against the oracle for a single step
from the same state and for short horizons (LES flow is chaotic, so long
horizons are compared statistically, not pointwise).  Pressure solves:
the FP64 residual norm reaches the same relative tolerance as the oracle's
SOR and the iteration counts agree within the check interval.
"""
import numpy as np
import pytest

import oracle
from oracle import les as ol
from paper_1711_04471_gb300 import inputs

pytestmark = pytest.mark.gpu

REL = 1e-5


@pytest.fixture(scope="module")
def G():
    import paper_1711_04471_gb300 as P
    P.build()
    from paper_1711_04471_gb300 import les
    oracle.lib()
    return les


def rel_l2(a, b, sl=None):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if sl is not None:
        a, b = a[sl], b[sl]
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


INT = (slice(1, -1), slice(1, -1), slice(1, -1))


def small_case(nx=32, ny=24, nz=16, seed=5):
    solid = inputs.les_buildings(nx, ny, nz, dx=4.0, seed=seed, cover=0.2, margin_cells=4)
    return nx, ny, nz, solid


# ------------------------------------------------------------- Poisson

def test_poisson_solve_matches_oracle_iterates(G):
    import torch
    nx, ny, nz, dx = 40, 32, 24, 4.0
    rng = np.random.default_rng(7)
    b = rng.standard_normal((nz, ny, nx))
    P = ol.make_params(nx, ny, nz, dx=dx)
    bo = ol.padded(P)
    ol.interior(bo)[:] = b.astype(np.float32)        # the GPU sees the FP32-rounded b
    po = ol.padded(P)
    rc, it_o, rr_o = ol.sor(P, bo, po, omega=1.8, tol=1e-6, max_iter=100000)
    assert rc == 0
    pg = torch.zeros((nz, ny, nx), dtype=torch.float32, device="cuda")
    bg = torch.from_numpy(b.astype(np.float32)).cuda()
    st, it_g, rr_g = G.poisson_solve(pg, bg, dx, omega=1.8, tol=1e-6, check_every=1)
    assert st == 0 and rr_g <= 1e-6
    assert abs(it_g - it_o) <= 1, (it_g, it_o)
    assert rel_l2(pg.cpu().numpy(), ol.interior(po)) <= 1e-5
    # check_every = 10: stops at the first multiple of 10 at or past the oracle's count
    pg.zero_()
    st, it10, rr10 = G.poisson_solve(pg, bg, dx, omega=1.8, tol=1e-6, check_every=10)
    assert st == 0 and rr10 <= 1e-6 and it10 % 10 == 0 and it_o - 1 <= it10 < it_o + 11


@pytest.mark.parametrize("shape", [(300, 16, 6), (257, 10, 5), (256, 6, 4), (512, 4, 2)])
def test_poisson_fixed_iterations_match_oracle_on_wide_rows(G, shape):
    """Rows wider than one block of the sweep and fold kernels: 150 and 129
    slots of a colour (the second an odd nx; both take the flat thread
    mapping), and 128 and 256 slots (one and two warps per row, the
    warp-per-row mapping).  300 fixed iterations with a fold and FP64
    residual in between (check every 50) against the oracle's iterates."""
    import torch
    nx, ny, nz = shape
    dx = 4.0
    rng = np.random.default_rng(nx)
    b = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    P = ol.make_params(nx, ny, nz, dx=dx)
    bo, po = ol.padded(P), ol.padded(P)
    ol.interior(bo)[:] = b
    ol.sor(P, bo, po, omega=1.8, tol=0.0, max_iter=300)
    for tol in (-1.0, 1e-30):       # paper mode (direct launches) and the graph with its checks
        pg = torch.zeros((nz, ny, nx), dtype=torch.float32, device="cuda")
        st, it, rr = G.poisson_solve(pg, torch.from_numpy(b).cuda(), dx, omega=1.8, tol=tol, max_iter=300,
                                     check_every=50)
        assert it == 300
        assert rel_l2(pg.cpu().numpy(), ol.interior(po)) <= 1e-5, tol
        assert abs(rr - ol.residual(P, bo, po)) <= 1e-3 * rr


def test_poisson_solve_reaches_fp64_accuracy(G):
    """The FP32 sweeps iterate on a correction of the FP64 pressure, so the
    residual keeps falling far below what FP32 storage of p alone allows."""
    import torch
    nx, ny, nz, dx = 24, 16, 20, 4.0
    rng = np.random.default_rng(8)
    b = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    pg = torch.zeros((nz, ny, nx), dtype=torch.float32, device="cuda")
    st, it, rr = G.poisson_solve(pg, torch.from_numpy(b).cuda(), dx, omega=1.9, tol=1e-11, check_every=20)
    assert st == 0 and rr <= 1e-11
    P = ol.make_params(nx, ny, nz, dx=dx)
    bo, po = ol.padded(P), ol.padded(P)
    ol.interior(bo)[:] = b
    ol.sor(P, bo, po, omega=1.9, tol=1e-13, max_iter=1000000)
    assert rel_l2(pg.cpu().numpy(), ol.interior(po)) <= 1e-7   # FP32 rounding of the returned p


def test_poisson_solve_edge_cases(G):
    import torch
    z = torch.zeros((4, 6, 5), dtype=torch.float32, device="cuda")
    st, it, rr = G.poisson_solve(z.clone(), z, 1.0)
    assert st == 0 and it == 0
    b = torch.ones((4, 6, 5), dtype=torch.float32, device="cuda")
    st, it, rr = G.poisson_solve(z.clone(), b, 1.0, tol=1e-12, max_iter=20, check_every=10)
    assert st == 1 and it == 20 and rr > 1e-12          # GBSW_NOT_CONVERGED is a status, not an error
    from paper_1711_04471_gb300._native import GBSWError
    with pytest.raises(GBSWError):
        G.poisson_solve(torch.zeros((4, 5, 5), device="cuda"), torch.zeros((4, 5, 5), device="cuda"), 1.0)  # odd ny


# ------------------------------------------------------------- LES step

def _gpu_from_oracle(G, s, nx, ny, nz, solid, **kw):
    g = G.LES(nx, ny, nz, solid, **kw)
    for name in ("u", "v", "w", "fuo", "fvo", "fwo", "gu", "gv", "gw"):
        g.set(name, getattr(s, name))
    g.set("p", s.p)
    g.step_count = s.step_count
    return g


def test_fixed_iteration_steps_match_oracle(G):
    """The paper's mode (les_set_fixed_iterations, 50 SOR iterations per
    step): two steps from rest, the second replaying the cached graph of the
    fixed-count solve, against the oracle stepping with exactly 50
    iterations (tolerance 0)."""
    nx, ny, nz, solid = small_case()
    P = ol.make_params(nx, ny, nz, tol=0.0, max_iter=50)
    s = ol.LESState(P, solid)
    with G.LES(nx, ny, nz, solid) as g:
        g.set_fixed_iterations(50)
        for step in range(2):
            st = g.step(1)[0]
            s.step(1)
            it_o, rr_o, _ = s.history[-1]
            assert st["iters"] == it_o == 50
            assert rel_l2(g.get("u"), s.u, INT) <= REL, step
            assert rel_l2(g.get("p"), s.p, INT) <= REL, step
            assert abs(st["rel_res"] - rr_o) <= 1e-3 * rr_o, step


def test_fixed_count_steps_reuse_the_stencil_bitwise(G):
    """Paper mode: the first residual of a fixed-count solve reuses the
    stencil that the previous solve's final residual stored (the pressure
    has not changed since).  Writing the pressure back between steps, which
    makes the solver form the stencil afresh, gives bitwise the same steps."""
    nx, ny, nz, solid = small_case(40, 32, 20, seed=9)
    out, res = [], []
    for rewrite in (False, True):
        with G.LES(nx, ny, nz, solid) as g:
            g.set_fixed_iterations(30)
            r = []
            for _ in range(4):
                r.append(g.step(1)[0]["rel_res"])
                if rewrite:
                    g.set("p", g.get("p"))
            out.append({n: g.get(n) for n in ("u", "v", "w", "p", "b")})
            res.append(r)
    for n in out[0]:
        assert np.array_equal(out[0][n][INT], out[1][n][INT]), n
    assert res[0] == res[1]


@pytest.mark.parametrize("warm", [0, 3])
def test_single_step_from_identical_state(G, warm):
    nx, ny, nz, solid = small_case()
    P = ol.make_params(nx, ny, nz, tol=1e-9)
    s = ol.LESState(P, solid).step(warm)
    with _gpu_from_oracle(G, s, nx, ny, nz, solid, tol=1e-9, check_every=5) as g:
        stats = g.step(1)
        s.step(1)
        for name in ("u", "v", "w", "fuo", "fvo", "fwo", "gu", "gv", "gw", "b"):
            assert rel_l2(g.get(name), getattr(s, name), INT) <= REL, name
        assert rel_l2(g.get("nut"), s.nut, INT) <= REL
        assert rel_l2(g.get("p"), s.p, INT) <= REL
    assert stats[0]["status"] == 0 and stats[0]["rel_res"] <= 1e-9
    it_o = s.history[-1][0]
    assert it_o - 1 <= stats[0]["iters"] < it_o + 6


def test_predicted_checks_keep_the_stopping_rule(G):
    """Predicted convergence checks (the default of an LES context): with
    check_every = 100 the solve loop runs chunks of 50 iterations and checks
    where the measured convergence rate puts the tolerance, at most 100
    iterations after the previous check.  Both variants stop at a check
    whose FP64 residual is within tol: the fixed interval at the first
    multiple of 100 past the oracle's count, the predicted one at a multiple
    of 50 within one interval of it; the pressure matches the oracle."""
    nx, ny, nz, solid = small_case()
    P = ol.make_params(nx, ny, nz, tol=1e-9)
    s = ol.LESState(P, solid).step(3)
    got = {}
    for predicted in (False, True):
        with _gpu_from_oracle(G, s, nx, ny, nz, solid, tol=1e-9, check_every=100) as g:
            if not predicted:
                g.set_check_prediction(False)
            st = g.step(1)[0]
            got[predicted] = (st, g.get("p"))
    s.step(1)
    it_o = s.history[-1][0]
    off, on = got[False][0], got[True][0]
    assert off["status"] == on["status"] == 0 and off["rel_res"] <= 1e-9 and on["rel_res"] <= 1e-9
    assert off["iters"] % 100 == 0 and it_o - 1 <= off["iters"] < it_o + 100, (off["iters"], it_o)
    assert on["iters"] % 50 == 0 and it_o - 1 <= on["iters"] < it_o + 100, (on["iters"], it_o)
    for predicted in (False, True):
        assert rel_l2(got[predicted][1], s.p, INT) <= REL, predicted


def test_ten_step_horizon_and_iteration_counts(G):
    nx, ny, nz, solid = small_case(40, 32, 20, seed=9)
    P = ol.make_params(nx, ny, nz)
    s = ol.LESState(P, solid).step(10)
    with G.LES(nx, ny, nz, solid, check_every=1) as g:
        stats = g.step(10)
        assert rel_l2(g.get("u"), s.u, INT) <= REL
        assert rel_l2(g.get("v"), s.v, INT) <= 10 * REL
        assert rel_l2(g.get("p"), s.p, INT) <= 10 * REL
    for st, (it_o, rr_o, rc) in zip(stats, s.history):
        assert st["status"] == 0 and st["rel_res"] <= 1e-6
        assert abs(st["iters"] - it_o) <= 2, (st["iters"], it_o)


def test_checkpoint_restart_is_bit_identical(G):
    nx, ny, nz, solid = small_case(32, 16, 12, seed=3)
    names = ("u", "v", "w", "p", "fuo", "fvo", "fwo", "gu", "gv", "gw")
    with G.LES(nx, ny, nz, solid) as a:
        a.step(6)
        ref = {n: a.get(n) for n in names}
    with G.LES(nx, ny, nz, solid) as b:
        b.step(3)
        ck = {n: b.get(n) for n in names}
        k = b.step_count
    with G.LES(nx, ny, nz, solid) as c:
        for n in names:
            c.set(n, ck[n])
        c.step_count = k
        c.step(3)
        for n in names:
            assert np.array_equal(c.get(n)[INT], ref[n][INT]), n


def test_field_copies_through_pinned_and_pageable_buffers_agree(G):
    """les_get_field / les_set_field copy a page-locked host buffer directly
    and a pageable one through the context's staging buffer: both move the
    same bytes, in both directions."""
    import ctypes as C

    import torch

    from paper_1711_04471_gb300 import _native as N
    nx, ny, nz, solid = small_case(32, 16, 12, seed=3)
    with G.LES(nx, ny, nz, solid) as g:
        g.step(2)
        for name in ("p", "u", "gu"):
            dt = np.float64 if name == "p" else np.float32
            pinned = g.get(name)                       # the binding's page-locked array
            assert torch.from_numpy(pinned).is_pinned()
            pageable = np.empty(pinned.shape, dt)
            N.check(N.lib().les_get_field(g._h, G.FIELDS[name], pageable.ctypes.data_as(C.c_void_p)), "get")
            assert np.array_equal(pinned, pageable), name
            new = pageable * 1.5 + 0.25                # written from pageable memory, read back pinned
            N.check(N.lib().les_set_field(g._h, G.FIELDS[name], new.ctypes.data_as(C.c_void_p)), "set")
            assert np.array_equal(g.get(name), new), name
            src = torch.from_numpy(pageable).pin_memory()   # written from pinned memory, read back pageable
            N.check(N.lib().les_set_field(g._h, G.FIELDS[name], C.c_void_p(src.data_ptr())), "set")
            back = np.empty(pinned.shape, dt)
            N.check(N.lib().les_get_field(g._h, G.FIELDS[name], back.ctypes.data_as(C.c_void_p)), "get")
            assert np.array_equal(back, pageable), name


def test_whole_state_checkpoint_restart_is_bit_identical(G):
    """les_get_state / les_set_state: a context restored from a checkpoint
    takes bitwise the steps the original takes."""
    nx, ny, nz, solid = small_case(32, 16, 12, seed=4)
    with G.LES(nx, ny, nz, solid) as a, G.LES(nx, ny, nz, solid) as b:
        a.step(3)
        ck = a.get_state()
        assert ck["step"] == 3
        a.step(3)
        want = a.get_state()
        b.set_state(ck)
        assert b.step_count == 3
        b.step(3)
        got = b.get_state()
    for n in G.LES.STATE:
        assert np.array_equal(got[n][INT], want[n][INT]), n
    assert got["step"] == want["step"] == 6


def test_no_buildings_and_minimal_sizes(G):
    """Without buildings the inflow is nearly divergence-free and b is at the
    level of FP32 rounding of the face velocities, so p is compared through
    the oracle's FP64 residual of the GPU's own b rather than pointwise."""
    for nx, ny, nz in [(2, 2, 2), (5, 4, 3), (33, 18, 7)]:
        P = ol.make_params(nx, ny, nz, tol=1e-8)
        solid = np.zeros((nz, ny, nx), np.uint8)
        s = ol.LESState(P, solid).step(2)
        with G.LES(nx, ny, nz, None, tol=1e-8, check_every=1) as g:
            st = g.step(2)
            assert rel_l2(g.get("u"), s.u, INT) <= REL, (nx, ny, nz)
            b = g.get("b").astype(np.float64)
            assert ol.residual(P, b, g.get("p")) <= 1.001e-8 or np.abs(b).max() < 1e-30
            assert all(x["status"] == 0 for x in st)


def test_argument_errors(G):
    from paper_1711_04471_gb300._native import GBSWError
    with pytest.raises(GBSWError):
        G.LES(8, 7, 4)                      # odd ny
    with pytest.raises(GBSWError) as e:
        G.LES(8, 8, 4, dt=1.0)              # CFL
    assert e.value.status == -4


def test_full_size_step(G):
    """256 x 256 x 128 with 20 % building cover: the GPU step against the
    oracle's subroutines applied to the same FP64-cast state, and the GPU
    pressure's FP64 residual recomputed by the oracle."""
    nx, ny, nz = 256, 256, 128
    solid = inputs.les_buildings(nx, ny, nz, dx=4.0, seed=1003)
    with G.LES(nx, ny, nz, solid, max_iter=20000) as g:
        stats = g.step(2)
        assert all(st["status"] in (0, 1) for st in stats)
        st_fields = {n: g.get(n).astype(np.float64) for n in ("u", "v", "w", "fuo", "fvo", "fwo", "gu", "gv", "gw")}
        p = g.get("p")
        stats3 = g.step(1)
        u3, b3, p3 = g.get("u"), g.get("b"), g.get("p")
    P = ol.make_params(nx, ny, nz)
    u, v, w = st_fields["u"], st_fields["v"], st_fields["w"]
    ol.velnw(P, p, u, v, w)
    ol.bondv1(P, u, v, w)
    fu, fv, fw = ol.velfg(P, u, v, w)
    ol.feedbf(P, solid, u, v, w, st_fields["gu"], st_fields["gv"], st_fields["gw"], fu, fv, fw)
    nt = ol.nut(P, u, v, w)
    ol.visc(P, u, v, w, nt, fu, fv, fw)
    ol.adam(P, False, u, v, w, fu, fv, fw, st_fields["fuo"], st_fields["fvo"], st_fields["fwo"])
    b = ol.rhs(P, u, v, w)
    assert rel_l2(u3, u, INT) <= REL
    assert rel_l2(b3, b, INT) <= 1e-4     # b is a difference of nearly equal face velocities
    res = ol.residual(P, b3.astype(np.float64), p3)
    # the device's FP64 residual of its pressure is what the oracle computes
    assert abs(res - stats3[0]["rel_res"]) <= 1e-3 * res, (res, stats3[0]["rel_res"])
    if stats3[0]["status"] == 0:
        assert res <= 1.0001e-6

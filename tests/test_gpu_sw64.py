"""The FP64 2DSW path (sw64_*, three kernels per step, every operation
rounded as written) against the FP64 oracle: the fields must be equal bit
for bit, wet/dry masks included, since both evaluate the same expressions
in the same order in IEEE double precision.  Only the volume, a sum in a
different order, is compared to rounding (1e-13 relative)."""
import numpy as np
import pytest

import oracle
from paper_1711_04471_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SW64():
    import paper_1711_04471_gb300 as P
    P.build()
    from paper_1711_04471_gb300.sw import SW64
    return SW64


def run_both(SW64, inp, nsteps):
    o = oracle.SWState(inp.params(), inp.H, inp.eta0).run(nsteps)
    with SW64(inp.params(), inp.H, inp.eta0) as g:
        g.step(nsteps)
        st = g.get_state()
        vol = g.volume()
    return o, st, vol


def assert_bitwise(o, st):
    assert np.array_equal(st["eta"], o.eta_i)
    assert np.array_equal(st["u"], o.u_f)
    assert np.array_equal(st["v"], o.v_f)
    assert np.array_equal(st["wet"], o.wet_i)


def test_hump_1000_steps_bitwise(SW64):
    inp = inputs.sw_hump()
    o, st, vol = run_both(SW64, inp, 1000)
    assert_bitwise(o, st)
    v_or, w_or = o.volume()
    assert vol[0] == pytest.approx(v_or, rel=1e-13) and vol[1] == pytest.approx(w_or, rel=1e-13)


@pytest.mark.parametrize("n,seed,steps", [(200, 7, 300), (160, 31, 500)])
def test_wetdry_bitwise(SW64, n, seed, steps):
    """Wet/dry bathymetry with dry land: masks and fields equal bit for bit
    (no margin certificate is needed when the arithmetic is identical)."""
    inp = inputs.sw_wetdry(n=n, seed=seed)
    o, st, vol = run_both(SW64, inp, steps)
    assert 0 < int(st["wet"].sum()) < n * n
    assert_bitwise(o, st)


def test_rectangular_ragged_and_paper_setup(SW64):
    """Odd, non-square grids across the 128-thread row blocks, and the
    paper's dx = 1 m, dt = 0.01 s setting."""
    for nx, ny in ((37, 23), (130, 9), (2, 2)):
        base = inputs.sw_wetdry(n=max(nx, ny), seed=nx + ny)
        H = np.ascontiguousarray(base.H[:ny, :nx])
        eta0 = np.ascontiguousarray(base.eta0[:ny, :nx])
        inp = inputs.SWInput(nx, ny, base.dx, base.dy, base.dt, H, eta0, hmin=base.hmin)
        o, st, _ = run_both(SW64, inp, 120)
        assert_bitwise(o, st)
    inp = inputs.sw_hump(n=200, dx=1.0, dt=0.01, sigma_cells=10.0)
    o, st, _ = run_both(SW64, inp, 200)
    assert_bitwise(o, st)


def test_lake_at_rest_and_errors(SW64):
    base = inputs.sw_wetdry(n=120, seed=3)
    eta0 = np.maximum(0.0, -base.H)
    inp = inputs.SWInput(base.nx, base.ny, base.dx, base.dy, base.dt, base.H, eta0, hmin=base.hmin)
    with SW64(inp.params(), inp.H, inp.eta0) as g:
        g.step(500)
        st = g.get_state()
    assert np.array_equal(st["eta"], eta0)
    assert not st["u"].any() and not st["v"].any()
    from paper_1711_04471_gb300._native import GBSWError
    p = inp.params()
    with pytest.raises(GBSWError):
        SW64(dict(p, dt=100.0), inp.H, inp.eta0)          # CFL
    with pytest.raises(ValueError):
        SW64(p, inp.H[:, :-1], inp.eta0)

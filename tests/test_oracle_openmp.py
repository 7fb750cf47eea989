"""The OpenMP build of the oracle (used only to time it on all host cores)
gives bitwise the same results as the serial build: its threads split only
the outer loops of the per-cell maps, and every sum runs serially in the
same order."""
import numpy as np

import oracle
from oracle import les
from paper_1711_04471_gb300 import inputs


def _sw_run(openmp, inp, nsteps):
    oracle.use_openmp(openmp)
    try:
        s = oracle.SWState(inp.params(), inp.H, inp.eta0).run(nsteps)
        return s.eta.copy(), s.u.copy(), s.v.copy(), s.margin, s.volume()
    finally:
        oracle.use_openmp(False)


def test_openmp_build_uses_several_threads():
    assert oracle.threads(openmp=False) == 1
    assert oracle.threads(4) == 4


def test_sw_openmp_bitwise_equal():
    oracle.threads(4)
    inp = inputs.sw_wetdry(n=96, seed=7)
    a = _sw_run(False, inp, 40)
    b = _sw_run(True, inp, 40)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    assert a[3] == b[3] and a[4] == b[4]


def test_les_openmp_bitwise_equal():
    oracle.threads(4)
    nx, ny, nz = 16, 12, 10
    solid = np.zeros((nz, ny, nx), np.uint8)
    solid[:4, 3:6, 5:8] = 1
    P = les.make_params(nx, ny, nz, tol=1e-9)
    out = []
    for omp in (False, True):
        oracle.use_openmp(omp)
        try:
            s = les.LESState(P, solid).step(2)
            out.append(({n: getattr(s, n).copy() for n in les.LESState.NAMES}, list(s.history)))
        finally:
            oracle.use_openmp(False)
    (fa, ha), (fb, hb) = out
    assert ha == hb                      # same SOR iteration counts and residuals, bit for bit
    for n in fa:
        assert np.array_equal(fa[n], fb[n]), n

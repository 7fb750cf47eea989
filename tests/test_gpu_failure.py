"""Failure detection without a GPU fault: bounded device waits give up and
report, bad inputs are refused on the host, NaN is reported by the FP64
reductions; the context stays usable afterwards."""
import numpy as np
import pytest

from paper_1711_04471_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_1711_04471_gb300 as P
    P.build()
    from paper_1711_04471_gb300 import _native as N
    return N.lib()


@pytest.mark.parametrize("which,budget", [(0, 2_000_000), (1, 20_000)])
def test_bounded_waits_time_out_and_context_survives(lib, which, budget):
    assert lib.gbsw_selftest_wait(which, budget) == -6          # GBSW_ERR_TIMEOUT
    from paper_1711_04471_gb300.sw import SW
    inp = inputs.sw_hump(n=32)
    with SW(inp.params(), inp.H, inp.eta0) as g:
        g.step(10)
        v, _ = g.volume()
    assert np.isfinite(v)


def test_selftest_rejects_bad_budget(lib):
    assert lib.gbsw_selftest_wait(0, 0) == -1
    assert lib.gbsw_selftest_wait(2, 10) == -1
    assert lib.gbsw_selftest_wait(1, 10**12) == -1


def test_solver_reports_not_converged_and_nonfinite_rhs(lib):
    import torch

    from paper_1711_04471_gb300.les import poisson_solve
    b = torch.ones((4, 6, 8), device="cuda")
    st, it, rr = poisson_solve(torch.zeros_like(b), b, 4.0, tol=1e-14, max_iter=10, check_every=5)
    assert st == 1 and it == 10
    b[1, 2, 3] = float("nan")
    from paper_1711_04471_gb300._native import GBSWError
    with pytest.raises(GBSWError) as e:
        poisson_solve(torch.zeros_like(b), b, 4.0, tol=1e-6, max_iter=10, check_every=5)
    assert e.value.status == -5


@pytest.mark.parametrize("d", [4, 5, 6, 7])
def test_sor_division_is_correctly_rounded(lib, d):
    """The sweep's division by the diagonal (rounded reciprocal plus one FMA
    correction) equals the IEEE division x / d bit for bit for every finite
    FP32 x of magnitude at least 2^-100 (SOR values never get near that)."""
    import ctypes as C
    counts = (C.c_ulonglong * 3)()
    assert lib.gbsw_selftest_sor_division(d, counts) == 0
    print(f"d = {d}: {counts[0]} mismatches for |x| >= 2^-100, {counts[1]} below, first {counts[2]:#x}")
    assert counts[0] == 0, (counts[0], hex(counts[2]))


def test_sor_division_selftest_rejects_bad_arguments(lib):
    import ctypes as C
    counts = (C.c_ulonglong * 3)()
    assert lib.gbsw_selftest_sor_division(3, counts) == -1
    assert lib.gbsw_selftest_sor_division(8, counts) == -1
    assert lib.gbsw_selftest_sor_division(6, None) == -1


def test_ensemble_barrier_timeout_is_reported(lib, monkeypatch):
    """GBSW_FAULT=sync_timeout gives the persistent ensemble kernel's grid
    barrier a zero spin budget: the first wait gives up, every block leaves,
    and the next syncing call reports GBSW_ERR_TIMEOUT.  A new ensemble
    without the injection then runs normally on the same context."""
    from paper_1711_04471_gb300.sw import SWBatch
    from paper_1711_04471_gb300._native import GBSWError
    members = [inputs.sw_ensemble_member(n, 1002, k) for k, n in enumerate((64, 96, 130, 200))]
    monkeypatch.setenv("GBSW_FAULT", "sync_timeout")
    b = SWBatch(members)
    b.set_tiling(2, 64)
    b.step(6)                      # three levels: two grid barriers
    with pytest.raises(GBSWError) as e:
        b.volumes()
    assert e.value.status == -6
    b.close()
    monkeypatch.delenv("GBSW_FAULT")
    with SWBatch(members) as ok:
        ok.set_tiling(2, 64)
        ok.step(6)
        vols, _ = ok.volumes()
    assert np.all(np.isfinite(vols))

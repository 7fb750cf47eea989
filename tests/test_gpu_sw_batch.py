"""The batched 2DSW ensemble (one persistent kernel, grid barriers between
fused levels) against the single-instance path and the FP64 oracle.

Per cell the arithmetic of a step does not depend on how steps are fused
or tiles are cut, so the ensemble must reproduce sw_step bit for bit, for
every tiling; a stale read across the grid barrier would break that.
"""
import numpy as np
import pytest

import oracle
from paper_1711_04471_gb300 import inputs
from sw_cases import fixed_shores

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import paper_1711_04471_gb300 as P
    P.build()
    from paper_1711_04471_gb300 import sw
    return sw


def members(count=10, seed=77):
    sizes = inputs.sw_ensemble_sizes(count, seed=seed, nmin=40, nmax=300)
    out = [inputs.sw_ensemble_member(int(n), seed, k) for k, n in enumerate(sizes)]
    # one non-square member and one tiny one
    out.append(inputs.SWInput(70, 33, 10.0, 10.0, 0.1, np.full((33, 70), 12.0),
                              0.2 * np.exp(-((np.arange(70)[None, :] - 30.0) ** 2) / 50.0) * np.ones((33, 1))))
    out.append(inputs.sw_hump(n=8))
    return out


def test_batch_equals_single_instances_bitwise(mods):
    ms = members()
    nsteps = 37  # 12 levels of 3 plus a one-step remainder level
    with mods.SWBatch(ms) as b:
        b.set_tiling(3, 64)
        b.step(nsteps)
        got = [b.get_state(k) for k in range(len(ms))]
        vols, _ = b.volumes()
    for k, m in enumerate(ms):
        with mods.SW(m.params(), m.H, m.eta0) as g:
            g.set_blocking(3)
            g.step(nsteps)
            ref = g.get_state()
            vref, _ = g.volume()
        for f in ("eta", "u", "v"):
            assert np.array_equal(got[k][f], ref[f]), (k, f)
        assert abs(vols[k] - vref) <= 1e-12 * abs(vref)


@pytest.mark.parametrize("T,rows", [(1, 32), (2, 128), (4, 16), (3, 1000)])
def test_tilings_agree_bitwise(mods, T, rows):
    ms = members(6, seed=5)
    with mods.SWBatch(ms) as a:
        a.set_tiling(3, 64)
        a.step(24)
        ref = [a.get_state(k) for k in range(len(ms))]
    with mods.SWBatch(ms) as b:
        b.set_tiling(T, rows)
        b.step(20)
        b.step(4)
        for k in range(len(ms)):
            s = b.get_state(k)
            for f in ("eta", "u", "v"):
                assert np.array_equal(s[f], ref[k][f]), (k, f, T, rows)


def test_separate_launches_match_persistent(mods):
    ms = members(5, seed=9)
    with mods.SWBatch(ms) as a, mods.SWBatch(ms) as b:
        a.step(30)
        b.step_separate(30)
        for k in range(len(ms)):
            sa, sb = a.get_state(k), b.get_state(k)
            for f in ("eta", "u", "v"):
                assert np.array_equal(sa[f], sb[f])


def test_batch_1000_steps_against_sw_step_and_oracle(mods):
    """1000 steps of an ensemble in the tiling the autotuner picks: every
    member equals the single-instance sw_step bit for bit, and every member
    whose oracle run certifies the wet/dry margin (min |h - hmin| > 1e-5 m
    over the run) matches the FP64 oracle: masks bit-exact, FP32 fields
    within 1e-5 relative L2.  Certified members: steep-shore wet/dry grids
    (sw_cases.fixed_shores, square and ragged) and all-wet humps; the
    moving-shore members of the workload recipe are checked through sw_step
    and, where their margin falls below 1e-5 m, by counting mask flips."""
    ms = [fixed_shores(72, 31), fixed_shores(150, 32, ny=97), fixed_shores(260, 33), fixed_shores(48, 34, ny=40),
          inputs.sw_hump(n=64), inputs.sw_hump(n=130)]
    ms += [inputs.sw_ensemble_member(int(n), 41, k)
           for k, n in enumerate(inputs.sw_ensemble_sizes(4, seed=41, nmin=40, nmax=300))]
    nsteps = 1000
    with mods.SWBatch(ms) as b:
        T, rows = b.autotune(trial_steps=8)
        b.step(nsteps)
        got = [b.get_state(k) for k in range(len(ms))]
        vols, _ = b.volumes()
    for k, m in enumerate(ms):
        # the wet mask as the kernels form it: FP32 H + eta > FP32 hmin
        got[k]["wet"] = ((m.H.astype(np.float32) + got[k]["eta"]) > np.float32(m.hmin)).astype(np.uint8)
    certified = 0
    for k, m in enumerate(ms):
        with mods.SW(m.params(), m.H, m.eta0) as g:
            g.set_blocking(T)
            g.step(nsteps)
            ref = g.get_state()
            vref, _ = g.volume()
        for f in ("eta", "u", "v", "wet"):
            assert np.array_equal(got[k][f], ref[f]), (k, f, T, rows)
        assert abs(vols[k] - vref) <= 1e-12 * abs(vref)   # both FP64 in a fixed order, not the same order
        o = oracle.SWState(m.params(), m.H, m.eta0).run(nsteps)
        rel = lambda a, b: np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
        if o.margin > 1e-5:
            certified += 1
            assert np.array_equal(got[k]["wet"], o.wet_i), k
            assert rel(got[k]["eta"], o.eta_i) <= 1e-5, k
            assert rel(got[k]["u"], o.u_f) <= 1e-5, k
            assert rel(got[k]["v"], o.v_f) <= 1e-5, k
        else:
            # moving shorelines: a few near-threshold cells may flip
            assert (got[k]["wet"] != o.wet_i).sum() <= 8, k
            assert rel(got[k]["eta"], o.eta_i) <= 1e-3, k
    assert certified >= 6


def test_autotune_keeps_state_and_caches(mods, tmp_path):
    ms = members(6, seed=13)
    cache = str(tmp_path / "tune.txt")
    with mods.SWBatch(ms) as a, mods.SWBatch(ms) as b:
        a.step(12)
        T, rows = b.autotune(trial_steps=8, cache_path=cache)
        assert 1 <= T <= 4 and rows in (32, 64, 128, 256)
        b.step(12)
        for k in range(len(ms)):
            for f in ("eta", "u", "v"):
                assert np.array_equal(a.get_state(k)[f], b.get_state(k)[f])
        T2, rows2 = b.autotune(trial_steps=8, cache_path=cache)
        assert (T2, rows2) == (T, rows)
    assert open(cache).read().count("\n") == 1

"""The seeded input recipes (paper_1711_04471_gb300/inputs.py) against what
they promise: the generator is SplitMix64 as published, the wet/dry
bathymetry has 15 % dry cells, ensemble sides are log-uniform in [64, 1024],
and the building masks cover 20 % of the ground away from the inflow and
outflow planes with the stated footprint and height ranges."""
import math

import numpy as np

from paper_1711_04471_gb300 import inputs

M64 = (1 << 64) - 1


def splitmix64_scalar(seed, n):
    """SplitMix64 (Steele, Lea & Flood 2014) transcribed with Python integers."""
    out, s = [], seed & M64
    for _ in range(n):
        s = (s + 0x9E3779B97F4A7C15) & M64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_matches_its_definition():
    assert splitmix64_scalar(0, 1)[0] == 0xE220A8397B1DCDAF       # first output from state 0
    for seed in (0, 1, 1001, inputs.derive_seed(2000, 7), M64):
        g = inputs.SplitMix64(seed)
        got = [int(x) for x in g.next_u64(5)] + [int(x) for x in g.next_u64(3)]
        assert got == splitmix64_scalar(seed, 8)
    u = inputs.SplitMix64(5).uniform(100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.005


def test_wetdry_bathymetry_has_fifteen_percent_dry_cells():
    inp = inputs.sw_wetdry(n=256, seed=1001)
    dry = np.mean(inp.H + inp.eta0 <= inp.hmin)
    assert 0.145 <= dry <= 0.155
    assert np.all(inp.eta0 >= -inp.H)
    wet = inp.H + inp.eta0 > inp.hmin
    assert np.abs(inp.eta0[wet]).max() <= 0.5 + 1e-12        # 0.5 m surface perturbation


def test_ensemble_sizes_are_log_uniform_in_range():
    n = inputs.sw_ensemble_sizes(512, seed=1002)
    assert n.min() >= 64 and n.max() <= 1024
    assert int((n.astype(np.int64) ** 2).sum()) == 87078320        # the ensemble benchmark's cell count
    logs = np.log(n / 64.0) / math.log(16.0)                      # U[0, 1) if log-uniform
    assert abs(logs.mean() - 0.5) < 0.05 and abs(logs.var() - 1.0 / 12.0) < 0.02


def test_building_mask_cover_margins_and_heights():
    nx, ny, nz, dx = 256, 128, 64, 4.0
    solid = inputs.les_buildings(nx, ny, nz, dx=dx, seed=1003)
    ground = solid[0].astype(bool)
    assert 0.20 <= ground.mean() < 0.26
    margin = max(2, nx // 16)
    assert not solid[:, :, :margin].any() and not solid[:, :, nx - margin:].any()
    heights = solid.sum(axis=0)                                  # cells per column
    assert heights.max() <= round(60.0 / dx) and heights[ground].min() >= round(10.0 / dx)
    # every column is a solid stack from the ground up
    assert np.all(np.diff(solid.astype(np.int8), axis=0) <= 0)

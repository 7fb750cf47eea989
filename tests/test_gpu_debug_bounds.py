"""The bounds-checked debug build on the GPU.

gbsw_selftest_bounds feeds the index test an index one past the end of a
buffer (no access is made): the violation is counted and reported.  Then the
2DSW kernels (streaming with several segment heights, the tile kernel, the
ensemble kernel), the SOR solve (warp-per-row and flat thread mappings) and
the UFLES predictor kernels (velnw, the fused predictor, the right-hand
side; whole and ragged tiles) and the learned warm start's grid transfers
run in the debug library in a child process:
no index leaves its buffer, and every result equals the product build's
bit for bit."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes as C, json, sys
import numpy as np
sys.path.insert(0, ROOT)
import paper_1711_04471_gb300 as P
P.build()
import torch
from paper_1711_04471_gb300 import _native as N, inputs
from paper_1711_04471_gb300.sw import SW, SWBatch
from paper_1711_04471_gb300.les import poisson_solve
out = {}
inp = inputs.sw_wetdry(n=150, seed=8)
for T, rows in [(3, 0), (2, 5), (6, 2), (2, -1), (3, -1), (1, -52), (3, -34), (3, -27)]:
    with SW(inp.params(), inp.H, inp.eta0) as g:
        g.set_tiling(T, rows)
        g.step(37)
        out[f"sw_{T}_{rows}"] = g.get_state()["eta"]
ms = [inputs.sw_ensemble_member(int(n), 7, k) for k, n in enumerate(inputs.sw_ensemble_sizes(5, seed=7, nmin=40, nmax=200))]
with SWBatch(ms) as b:
    b.set_tiling(3, 32)
    b.step(20)
    out["batch"] = b.get_state(2)["eta"]
for nx, ny, nz in [(256, 64, 9), (150, 40, 7)]:
    gen = torch.Generator(device="cuda").manual_seed(1)
    bb = torch.randn((nz, ny, nx), device="cuda", generator=gen)
    p = torch.zeros_like(bb)
    poisson_solve(p, bb, 4.0, tol=-1.0, max_iter=60, check_every=50)
    out[f"sor_{nx}"] = p.cpu().numpy()
from paper_1711_04471_gb300.les import LES
for nx, ny, nz in [(40, 32, 20), (37, 30, 11)]:   # whole and ragged tiles, chunks of planes
    solid = inputs.les_buildings(nx, ny, nz, dx=4.0, seed=5, cover=0.2, margin_cells=4)
    with LES(nx, ny, nz, solid) as g:
        g.set_fixed_iterations(20)
        g.step(3, stats=False)
        for name in ("u", "v", "w", "p", "nut", "b"):
            out[f"les_{nx}_{name}"] = g.get(name)[1:-1, 1:-1, 1:-1].copy()
from paper_1711_04471_gb300.unet import UNet
solid = inputs.les_buildings(64, 64, 32, dx=4.0, seed=6, cover=0.2, margin_cells=4)
with UNet(seed=0) as net, LES(64, 64, 32, solid) as g:   # the learned warm start's grid transfers
    g.set_warm_start(net)
    g.set_fixed_iterations(20)
    g.step(2, stats=False)
    out["les_ws_p"] = g.get("p")[1:-1, 1:-1, 1:-1].copy()
v = C.c_longlong()
st = N.lib().gbsw_debug_bounds(C.byref(v))
np.savez(OUT, **out)
print(json.dumps({"status": st, "violations": v.value}))
"""


def _run(tmp_path, debug):
    path = str(tmp_path / ("debug.npz" if debug else "product.npz"))
    env = dict(os.environ)
    env.pop("GBSW_DEBUG_BOUNDS", None)
    if debug:
        env["GBSW_DEBUG_BOUNDS"] = "1"
    code = f"ROOT = {ROOT!r}\nOUT = {path!r}\n" + CHILD
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), np.load(path)


def test_index_test_reports_a_violation():
    import paper_1711_04471_gb300 as P
    P.build()
    from paper_1711_04471_gb300 import _native as N
    assert N.lib().gbsw_selftest_bounds() == -7          # GBSW_ERR_DEVICE_BOUNDS


def test_debug_build_finds_no_violation_and_matches_product(tmp_path):
    rep_p, prod = _run(tmp_path, False)
    rep_d, dbg = _run(tmp_path, True)
    assert rep_p == {"status": 0, "violations": -1}      # the product build has no checks
    assert rep_d == {"status": 0, "violations": 0}
    for k in prod.files:
        assert np.array_equal(prod[k], dbg[k]), k

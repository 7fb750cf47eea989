"""Stored fixtures under tests/golden/.

paper_setups.json holds numbers printed in the paper (each entry names its
section); the tests check that the oracle and the library defaults follow
them.  oracle_*.json hold oracle values written by tests/golden/make_golden.py
(which calls only oracle/); the oracle must keep reproducing them (the C
oracle is built with -ffp-contract=off, so x86-64 and aarch64 hosts agree to
rounding)."""
import json
import os
import re
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")
sys.path.insert(0, GOLDEN)


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def close(a, b, rel=1e-12, abs_=1e-13):
    return abs(a - b) <= rel * abs(b) + abs_


def test_oracle_reproduces_stored_sw_hump():
    import make_golden
    want = load("oracle_sw_hump.json")
    got = make_golden.sw_hump_case()
    for key in ("eta", "u"):
        for (j, i, a), (j2, i2, b) in zip(got[key], want[key]):
            assert (j, i) == (j2, i2) and close(a, b), (key, j, i, a, b)
    assert close(got["volume_m3"], want["volume_m3"], rel=1e-14)
    assert close(got["wet_volume_m3"], want["wet_volume_m3"], rel=1e-14)


def test_oracle_reproduces_stored_les_step():
    import make_golden
    want = load("oracle_les_16x16x8.json")
    got = make_golden.les_case()
    assert got["status"] == want["status"] == 0
    assert got["sor_iterations"] == want["sor_iterations"]
    assert got["rel_res"] <= 1e-10
    for key in ("p", "u", "w"):
        for a, b in zip(got[key], want[key]):
            assert a[:3] == b[:3] and close(a[3], b[3], rel=1e-10, abs_=1e-12), (key, a, b)


def test_ufles_setup_follows_the_paper():
    """Sec. 6.3.2: 1.2 km over 300 cells is the 4 m grid spacing, and the time
    step is 0.025 s: the library's and the oracle's defaults."""
    from oracle import les as ol
    from paper_1711_04471_gb300 import les
    s = load("paper_setups.json")["ufles"]
    dx = s["domain_m"][0] / s["grid"][0]
    assert dx == les.DEFAULTS["dx"] == ol.DEFAULTS["dx"] == 4.0
    assert s["dt_s"] == les.DEFAULTS["dt"] == ol.DEFAULTS["dt"]


def test_oracle_step_calls_the_subroutines_in_the_paper_order():
    """Sec. 6.3.1 lists the seven subroutines of a UFLES step in order; the
    oracle's step runs them in that order ("les" is the eddy viscosity and
    its stress divergence; "press" the right-hand side and the SOR solve)."""
    order = load("paper_setups.json")["ufles"]["subroutine_order"]
    src = open(os.path.join(os.path.dirname(HERE), "oracle", "les_oracle.c")).read()
    body = src[src.index("int oracle_les_step("):]
    body = body[:body.index("\n}\n")]
    calls = re.findall(r"oracle_les_(\w+)\(", body)[1:]
    names = {"nut": "les", "visc": "les", "rhs": "press", "sor": "press"}
    seq = []
    for c in calls:
        n = names.get(c, c)
        if not seq or seq[-1] != n:
            seq.append(n)
    assert seq == order


def test_paper_2dsw_setup_in_the_oracle():
    """Sec. 6.2: dx = 1 m and dt = 0.01 s on the smallest printed grid (500^2):
    the gravity-wave Courant number of the 10 m basin is about 0.1, and the
    oracle conserves volume over 20 steps."""
    import oracle
    from paper_1711_04471_gb300 import inputs
    s = load("paper_setups.json")["sw2d"]
    n = s["sizes"][0]
    inp = inputs.sw_hump(n=n, dx=s["dx_m"], dt=s["dt_s"], sigma_cells=n / 20.0)
    assert np.sqrt(9.81 * 11.0) * s["dt_s"] / s["dx_m"] < 0.15
    o = oracle.SWState(inp.params(), inp.H, inp.eta0)
    v0, _ = o.volume()
    o.run(20)
    v1, _ = o.volume()
    assert abs(v1 - v0) / v0 <= 1e-12
    assert np.all(np.isfinite(o.eta_i))

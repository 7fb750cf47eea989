"""Write the stored oracle values under tests/golden/ (calls only oracle/).

    python tests/golden/make_golden.py

oracle_sw_hump.json: the FP64 2DSW oracle on the 100 x 100 hump basin
(10 m deep, dx = 10 m, dt = 0.1 s, 1 m hump of sigma 5 cells at the centre,
Shapiro eps = 0.05) after 200 steps, sampled at fixed cells and faces.
oracle_les_16x16x8.json: one FP64 UFLES step on a 16 x 16 x 8 grid with one
building block, SOR to 1e-10, sampled likewise.

The stored values pin the oracle against later changes of its own code: a
change of its arithmetic must come with regenerated values and a commit
message naming the passage (or its reading) that justifies it.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

SW_CELLS = [(50, 50), (49, 50), (50, 70), (10, 10), (0, 0), (99, 99), (25, 75)]     # (j, i) of eta
SW_UFACES = [(50, 50), (50, 60), (20, 30), (50, 0), (50, 100)]                    # (j, i) of u (east faces)
LES_CELLS = [(4, 8, 8), (1, 1, 1), (8, 16, 16), (4, 2, 14), (6, 12, 3)]           # padded (k, j, i)


def les_solid():
    s = np.zeros((8, 16, 16), np.uint8)
    s[0:4, 6:10, 6:9] = 1          # one block, 4 cells tall
    return s


def sw_hump_case():
    import oracle
    from paper_1711_04471_gb300 import inputs
    inp = inputs.sw_hump(n=100)
    o = oracle.SWState(inp.params(), inp.H, inp.eta0).run(200)
    vol, wet_vol = o.volume()
    return {
        "eta": [[j, i, float(o.eta_i[j, i])] for j, i in SW_CELLS],
        "u": [[j, i, float(o.u_f[j, i])] for j, i in SW_UFACES],
        "volume_m3": vol, "wet_volume_m3": wet_vol,
    }


def les_case():
    from oracle import les as ol
    P = ol.make_params(16, 16, 8, tol=1e-10)
    st = ol.LESState(P, les_solid()).step(1)
    it, rr, rc = st.history[-1]
    return {
        "p": [[k, j, i, float(st.p[k, j, i])] for k, j, i in LES_CELLS],
        "u": [[k, j, i, float(st.u[k, j, i])] for k, j, i in LES_CELLS],
        "w": [[k, j, i, float(st.w[k, j, i])] for k, j, i in LES_CELLS],
        "sor_iterations": it, "rel_res": rr, "status": rc,
    }


def main():
    sw = {"_comment": "FP64 2DSW oracle, 100x100 hump basin, 200 steps; written by tests/golden/make_golden.py",
          "steps": 200, **sw_hump_case()}
    with open(os.path.join(HERE, "oracle_sw_hump.json"), "w") as f:
        json.dump(sw, f, indent=1)
        f.write("\n")
    les = {"_comment": "FP64 UFLES oracle, 16x16x8 grid, one block, one step, SOR to 1e-10; written by "
                       "tests/golden/make_golden.py", **les_case()}
    with open(os.path.join(HERE, "oracle_les_16x16x8.json"), "w") as f:
        json.dump(les, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()

"""2DSW test cases shared by the GPU parity tests (not collected itself)."""
import numpy as np

from paper_1711_04471_gb300 import inputs


def fixed_shores(n, seed, ny=None, land=5.0, min_depth=1.5):
    """The 4096^2 workload's recipe (32 Gaussian hills scaled so 15 % of the
    cells are dry, a 0.5 m random-phase surface) on an n x n grid, cut to ny
    rows, with steep shores: every dry cell becomes land `land` m above the
    datum and every wet cell is at least `min_depth` deep.  Waves then run
    along fixed shorelines, so the wet/dry face rule and the masked filter
    act at every shoreline face in every step while no cell changes state:
    the oracle's margin certificate (min over the run of |h - hmin|) is the
    dry cells' 0.05 m for any number of steps."""
    base = inputs.sw_wetdry(n=n, seed=seed)
    ny = n if ny is None else ny
    dry = (base.H + base.eta0 <= base.hmin)[:ny]
    H = np.where(dry, -land, np.maximum(base.H[:ny], min_depth))
    eta = np.where(dry, land, base.eta0[:ny])
    return inputs.SWInput(base.nx, ny, base.dx, base.dy, base.dt, H, np.maximum(eta, -H), hmin=base.hmin)

"""sw_volume_noalloc: the volume reduction for callers that cannot allocate
device memory (for example because their own memory pool owns the whole
GPU, or because an allocation that may synchronise the device is not
allowed inside their time loop).  It keeps its partial sums in a fixed
array inside the library and runs the same kernels in the same sum order
as sw_volume, so it must give bitwise what sw_volume gives, and repeated
calls must leave the device's free memory unchanged.

This file is collected last on purpose; it also passes when run alone.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1711_04471_gb300 import inputs

pytestmark = pytest.mark.gpu

def _fields(inp, pitch_extra=7):
    """FP32 device copies of H and eta, in the layout the C ABI expects,
    with a row pitch wider than nx."""
    import torch
    eta = np.maximum(inp.eta0, -inp.H)
    pitch = inp.nx + pitch_extra
    Hd = torch.zeros((inp.ny, pitch), dtype=torch.float32)
    Ed = torch.zeros((inp.ny, pitch), dtype=torch.float32)
    Hd[:, :inp.nx] = torch.from_numpy(inp.H.astype(np.float32))
    Ed[:, :inp.nx] = torch.from_numpy(eta.astype(np.float32))
    return Hd.cuda(), Ed.cuda(), pitch


def _noalloc(L, inp, Hd, Ed, pitch, out):
    import torch
    st = L.sw_volume_noalloc(inp.nx, inp.ny, pitch, inp.dx, inp.dy, inp.hmin,
                             C.c_void_p(Hd.data_ptr()), C.c_void_p(Ed.data_ptr()),
                             C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, st
    torch.cuda.synchronize()
    return out.cpu().numpy().copy()


def test_noalloc_volume_matches_sw_volume_twice_in_a_row():
    import torch

    import paper_1711_04471_gb300 as P
    P.build()
    from paper_1711_04471_gb300 import _native
    from paper_1711_04471_gb300.sw import SW
    L = _native.lib()
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    for inp in (inputs.sw_wetdry(n=300, seed=5), inputs.sw_hump(n=130)):
        with SW(inp.params(), inp.H, inp.eta0) as g:
            ref_vol, ref_wet = g.volume()
        Hd, Ed, pitch = _fields(inp)
        _noalloc(L, inp, Hd, Ed, pitch, out)           # warm-up: loads the module, looks up the scratch array
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            got = _noalloc(L, inp, Hd, Ed, pitch, out)
            assert got[0] == ref_vol and got[1] == ref_wet and got[2] == 0.0
        assert torch.cuda.mem_get_info()[0] == free0    # nothing was allocated on the device


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch

    from paper_1711_04471_gb300 import _native
    L = _native.lib()
    buf = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    p = C.c_void_p(buf.data_ptr())
    o = C.c_void_p(out.data_ptr())
    assert L.sw_volume_noalloc((1 << 20) + 1, 2, (1 << 20) + 1, 1.0, 1.0, 0.05, p, p, o, None) == -1
    assert L.sw_volume_noalloc(4, 0, 4, 1.0, 1.0, 0.05, p, p, o, None) == -1
    assert L.sw_volume_noalloc(4, 2, 3, 1.0, 1.0, 0.05, p, p, o, None) == -1
    assert L.sw_volume_noalloc(4, 2, 4, 1.0, 1.0, 0.05, None, p, o, None) == -1

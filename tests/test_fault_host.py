"""Host-side fault injection (GBSW_FAULT=alloc): every create call of the
library reports GBSW_ERR_OOM, as it would on a failed device allocation,
before it touches a device, so this runs without a GPU."""
import numpy as np
import pytest

from paper_1711_04471_gb300 import inputs

OOM = -3


@pytest.fixture
def lib(monkeypatch):
    import paper_1711_04471_gb300 as P
    P.build()
    from paper_1711_04471_gb300 import _native as N
    N.lib()
    monkeypatch.setenv("GBSW_FAULT", "alloc")
    return N


def test_create_calls_report_out_of_memory(lib):
    from paper_1711_04471_gb300.les import LES
    from paper_1711_04471_gb300.sw import SW, SW64, SWBatch
    from paper_1711_04471_gb300.unet import UNet
    inp = inputs.sw_hump(n=16, sigma_cells=2.0)
    makers = [lambda: SW(inp.params(), inp.H, inp.eta0), lambda: SW64(inp.params(), inp.H, inp.eta0),
              lambda: SWBatch([inp, inp]), lambda: LES(16, 8, 4), lambda: UNet(seed=0)]
    for make in makers:
        with pytest.raises(lib.GBSWError) as e:
            make()
        assert e.value.status == OOM


def test_argument_errors_still_come_first(lib):
    """Bad arguments are refused before any injected allocation failure."""
    from paper_1711_04471_gb300.sw import SW
    inp = inputs.sw_hump(n=16, sigma_cells=2.0)
    H = inp.H.copy()
    H[0, 0] = np.nan
    with pytest.raises(lib.GBSWError) as e:
        SW(inp.params(), H, inp.eta0)
    assert e.value.status == -1

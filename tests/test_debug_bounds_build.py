"""The bounds-checked debug build (libgbsw_debug.so, GBSW_DEBUG_BOUNDS=1)
compiles for sm_103a from the same sources and exports the same C ABI
(no GPU needed)."""
import subprocess

from test_abi import declared_functions


def test_debug_build_exports_every_declared_symbol():
    import paper_1711_04471_gb300 as P
    lib = P.build(debug=True)
    assert lib.endswith("libgbsw_debug.so")
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert not sorted(declared_functions() - exported)

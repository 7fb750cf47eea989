"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/*.h (no GPU needed: nothing is computed)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.add(name)
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("sw_create", "sw_step", "sw_volume", "sw_get_state", "sw_set_state", "sw_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_1711_04471_gb300 as P
    lib = P.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = sorted(declared_functions() - exported)
    assert not missing, missing


def test_library_loads_without_gpu():
    from paper_1711_04471_gb300 import _native
    L = _native.lib()
    assert L.gbsw_version() >= 100
    assert L.gbsw_status_string(-4) == b"CFL condition violated"


def test_product_path_has_no_oracle_import():
    """The package never imports the oracle (it is test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_1711_04471_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True) + \
            glob.glob(os.path.join(pkg, "csrc", "*")):
        txt = open(f, errors="ignore").read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, flags=re.M), f
        assert "liboracle" not in txt and "oracle/" not in txt, f

"""The C-ABI library loads and exports every entry point that include/cr.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b(cr_[A-Za-z0-9_]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def cudalib():
    from paper_1308_5299_gb300 import build, binding
    build.build()
    return ctypes.CDLL(binding.LIB_PATH)


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ["cr_plan_create", "cr_plan_destroy", "cr_sht_synth", "cr_sht_adjoint", "cr_apply_A"]:
        assert must in names


def test_library_exports_every_declared_symbol(cudalib):
    missing = [n for n in declared_symbols() if not hasattr(cudalib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    from paper_1308_5299_gb300 import binding
    assert set(declared_symbols()) <= set(binding._SIGS)


def test_params_struct_size_matches_header():
    """The Python mirror of cr_params has the C layout (checked through a tiny
    C program compiled against the header)."""
    import subprocess
    import tempfile
    from paper_1308_5299_gb300 import binding
    src = '#include <stdio.h>\n#include <stddef.h>\n#include "cr.h"\nint main(){printf("%zu %zu %zu\\n", sizeof(cr_params), offsetof(cr_params, cl), offsetof(cr_params, stream));return 0;}\n'
    with tempfile.TemporaryDirectory() as d:
        open(os.path.join(d, "t.c"), "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), os.path.join(d, "t.c"), "-o", os.path.join(d, "t")])
        out = subprocess.check_output([os.path.join(d, "t")]).decode().split()
    P = binding.cr_params
    assert int(out[0]) == ctypes.sizeof(P)
    assert int(out[1]) == P.cl.offset
    assert int(out[2]) == P.stream.offset

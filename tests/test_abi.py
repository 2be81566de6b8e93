"""The C-ABI library builds for sm_103a, loads on a CPU-only host, and exports every symbol
include/chem.h declares (no compute calls here)."""
import ctypes
import os
import re

from conftest import ROOT


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            for mt in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
                names.add(mt.group(1))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2402_18858_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert {"chem_load_mech", "chem_rates", "chem_step_di", "thermo_props"} <= names
    for nm in sorted(names):
        assert hasattr(lib, nm), nm


def test_load_errors_without_gpu():
    """Parsing errors are reported through the ABI before any device work."""
    from paper_2402_18858_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.chem_load_mech.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
    lib.chem_last_error.restype = ctypes.c_char_p
    h = ctypes.c_void_p()
    rc = lib.chem_load_mech(os.path.join(ROOT, "tests", "golden", "unbalanced.mech").encode(), ctypes.byref(h))
    assert rc == -2 and not h.value
    assert b"balanced" in lib.chem_last_error()
    rc = lib.chem_load_mech(b"/nonexistent/x.mech", ctypes.byref(h))
    assert rc == -2

"""The C-ABI library loads and exports every entry point include/fdtd.h declares (CPU only)."""
import os
import re

from paper_1710_06829_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "fdtd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_expected_entry_points():
    assert declared_functions() == sorted(L.EXPORTS)


def test_library_loads_and_exports_all_symbols():
    lib = L.load()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    import ctypes as C
    assert C.sizeof(L.fdtd_grid) == 6 * 4 + 8 + 8
    assert C.sizeof(L.fdtd_coeffs) == 12 * 8
    assert C.sizeof(L.fdtd_source) == 8 + 7 * 8
    assert C.sizeof(L.fdtd_probe) == 8 + 8 + 8

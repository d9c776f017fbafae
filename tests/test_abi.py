"""The C-ABI library loads and exports every entry point include/fdtd.h declares (CPU only)."""
import os
import re

import pytest

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
    assert C.sizeof(L.fdtd_source) == 8 + 7 * 8 + 3 * 8
    assert C.sizeof(L.fdtd_probe) == 8 + 8 + 8
    assert C.sizeof(L.fdtd_species) == 6 * 8 + 8 + 2 * 8


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """sizeof and every field offset of the header's structs, as gcc lays them out, equal the
    binding's ctypes layout."""
    import ctypes as C
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    structs = {"fdtd_grid": L.fdtd_grid, "fdtd_coeffs": L.fdtd_coeffs,
               "fdtd_source": L.fdtd_source, "fdtd_probe": L.fdtd_probe,
               "fdtd_species": L.fdtd_species}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fdtd.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    inc = os.path.join(ROOT, "include")
    subprocess.run(["gcc", "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    got = dict(zip(out[0::2], map(int, out[1::2])))
    for name, cls in structs.items():
        assert got[name] == C.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[f"{name}.{fname}"] == getattr(cls, fname).offset, (name, fname)

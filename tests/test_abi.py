"""The C ABI library builds for sm_103a, loads, and exports every entry point declared in
include/hrt.h (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

from paper_1112_1071_gb300 import build, hrt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hrt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hrt_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = _declared()
    for must in ["hrt_create", "hrt_destroy", "hrt_set_grid_cartesian", "hrt_set_grid_spherical", "hrt_set_density",
                 "hrt_set_dust", "hrt_add_point_source", "hrt_set_cell_source", "hrt_set_peeloff",
                 "hrt_run_iteration", "hrt_get_temperature", "hrt_get_sed", "hrt_get_image", "hrt_batch_create",
                 "hrt_batch_run"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared()) <= set(hrt.exported_symbols())
    lib.hrt_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.hrt_version()


def test_binding_refuses_to_run_without_library(tmp_path):
    import pytest
    saved = hrt._lib
    hrt._lib = None
    try:
        with pytest.raises(ImportError):
            hrt.load(str(tmp_path / "missing.so"))
    finally:
        hrt._lib = saved


def test_binding_structs_have_the_header_layout(tmp_path):
    """The ctypes mirrors of hrt_run_params and hrt_iter_stats have the C compiler's size and
    field offsets for the declarations in include/hrt.h (a stale field would corrupt silently)."""
    import shutil
    import subprocess

    import pytest

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [hrt.hrt_run_params, hrt.hrt_iter_stats]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hrt.h"', "int main(void) {"]
    for S in structs:
        lines.append(f'printf("{S.__name__} size %zu\\n", sizeof({S.__name__}));')
        for name, _ in S._fields_:
            lines.append(f'printf("{S.__name__} {name} %zu\\n", offsetof({S.__name__}, {name}));')
    lines += ["return 0;", "}"]
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for row in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, field, value = row.split()
        got[(s, field)] = int(value)
    for S in structs:
        assert got[(S.__name__, "size")] == ctypes.sizeof(S), S.__name__
        for name, _ in S._fields_:
            assert got[(S.__name__, name)] == getattr(S, name).offset, (S.__name__, name)
    # and every field the header declares has a mirror
    body = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "hrt.h")).read(), flags=re.S)
    for S in structs:
        decl = re.search(r"typedef struct \{([^}]*)\}\s*" + S.__name__ + ";", body).group(1)
        names = re.findall(r"(\w+)\s*(?:,|;)", decl)
        assert sorted(names) == sorted(n for n, _ in S._fields_), S.__name__

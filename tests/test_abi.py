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

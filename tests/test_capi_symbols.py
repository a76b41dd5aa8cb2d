"""The C-ABI library builds, loads and exports every entry point that
include/ih.h declares (no GPU needed, nothing is computed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ih.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ih_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ih_create", "ih_build", "ih_query_rects", "ih_query_weighted", "ih_destroy"):
        assert n in names


def test_library_exports_all_declared(ihlib):
    lib = ctypes.CDLL(ihlib.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(ihlib.C_SYMBOLS) == sorted(_declared())


def test_struct_layouts_match_header(ihlib):
    # ih_frame: 4 int32, 2 pointers, int64, 3 int32 (+4 padding) -> 56 bytes on LP64
    assert ctypes.sizeof(ihlib.ih_frame) == 56
    assert ctypes.sizeof(ihlib.ih_frame_info) == 56
    assert ctypes.sizeof(ihlib.ih_batch_queries) == 56
    assert ctypes.sizeof(ihlib.ih_config) == 24


def test_binding_refuses_missing_library(tmp_path):
    from paper_1711_01656_gb300 import ih
    saved = ih._lib
    ih._lib = None
    try:
        with pytest.raises(ImportError):
            ih.load_library(str(tmp_path / "absent.so"))
    finally:
        ih._lib = saved

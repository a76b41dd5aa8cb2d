"""The C-ABI library builds, loads and exports every entry point that
include/ih.h declares (no GPU needed, nothing is computed)."""
import ctypes
import os
import re
import subprocess

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


STRUCTS = ["ih_channel", "ih_frame", "ih_config", "ih_frame_info", "ih_kernel_stat", "ih_batch_queries",
           "ih_server_config", "ih_request", "ih_completion"]


def test_struct_layouts_match_header(ihlib, tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    that a C compiler gives the structure of include/ih.h."""
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ih.h"', "int main(void) {"]
    for name in STRUCTS:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for field, _ in getattr(ihlib, name)._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, field, name, field))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    c = dict(l.split() for l in subprocess.check_output([str(exe)], text=True).splitlines())
    for name in STRUCTS:
        st = getattr(ihlib, name)
        assert int(c[name]) == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert int(c["%s.%s" % (name, field)]) == getattr(st, field).offset, (name, field)


def test_binding_refuses_missing_library(tmp_path):
    from paper_1711_01656_gb300 import ih
    saved = ih._lib
    ih._lib = None
    try:
        with pytest.raises(ImportError):
            ih.load_library(str(tmp_path / "absent.so"))
    finally:
        ih._lib = saved

"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/gwns.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gwns.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|double|const char \*)\s*\*?\s*(ns_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("ns_init", "ns_step", "ns_result", "ns_free", "ns_eval_lnl", "ns_strerror"):
        assert required in names
    assert len(names) >= 15


def test_library_builds_and_exports_every_symbol():
    from paper_2509_24949_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    lib.ns_strerror.restype = ctypes.c_char_p
    assert lib.ns_strerror(0) == b"ok"
    assert lib.ns_strerror(-3).startswith(b"k outside")
    # argument validation happens before any device work
    lib.ns_init.restype = ctypes.c_int
    assert lib.ns_init(None, None, None, None, None, None) == -1


def test_binding_refuses_to_run_without_library(tmp_path, monkeypatch):
    import paper_2509_24949_gb300 as g
    monkeypatch.setattr(g._build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(g, "_LIB", None)
    with pytest.raises(ImportError):
        g.lib()

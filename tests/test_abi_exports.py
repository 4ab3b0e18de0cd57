"""The C-ABI library builds for sm_103a, loads, and exports every function include/snsweep.h
declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "snsweep.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sn_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("sn_create", "sn_set_mesh", "sn_build_graph", "sn_sweep", "sn_moment", "sn_source_iterate"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1810_11080_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    lib = ctypes.CDLL(b.LIB)
    for n in declared_functions():
        assert hasattr(lib, n), n
    from paper_1810_11080_gb300 import EXPORTED
    assert sorted(EXPORTED) == declared_functions()


def test_binding_refuses_to_run_without_library(tmp_path):
    from paper_1810_11080_gb300 import _lib
    with pytest.raises(ImportError):
        _lib.load(str(tmp_path / "missing.so"))

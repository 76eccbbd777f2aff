"""The C-ABI library loads and exports every function include/swepi.h
declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "swepi.h")).read()
    return sorted(set(re.findall(r"\b(sw_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_boundary_calls():
    names = declared()
    for call in ("sw_init", "sw_rhs", "sw_jvp", "sw_kiops_phi", "sw_epi_step", "sw_free"):
        assert call in names


def test_library_exports_every_declared_symbol():
    from paper_2101_05617_gb300 import build as b
    if not os.path.exists(b.LIB):
        b.build()
    lib = ctypes.CDLL(b.LIB)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2101_05617_gb300 import swepi
    assert sorted(swepi.EXPORTED) == sorted(n for n in declared())


def test_status_strings_without_gpu():
    from paper_2101_05617_gb300 import swepi
    assert swepi.sw_status_str(0) == "ok"
    assert "invalid" in swepi.sw_status_str(-1)


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2101_05617_gb300 import swepi
    monkeypatch.setattr(swepi, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(swepi, "_lib", None)
    with pytest.raises(ImportError):
        swepi.lib()

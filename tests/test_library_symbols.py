"""The C ABI library builds for sm_103a, loads without a GPU and exports every
function include/sbt.h declares (no compute calls here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sbt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sbt_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    from paper_2207_03936_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    import importlib
    from paper_2207_03936_gb300 import sbt
    monkeypatch.setattr(sbt, "LIB", str(tmp_path / "absent.so"))
    monkeypatch.setattr(sbt, "_lib", None)
    import pytest
    with pytest.raises(ImportError):
        sbt.lib()
    importlib.reload(sbt)

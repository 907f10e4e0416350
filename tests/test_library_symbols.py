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


def test_create_rejects_invalid_geometry_and_config_before_any_cuda_call():
    """Argument checks of sbt_create run on the host before any CUDA call, so
    they answer SBT_ERR_ARG with a reason even where no GPU exists."""
    import numpy as np
    from paper_2207_03936_gb300 import sbt
    L = sbt.lib()
    mz = np.linspace(750, -290, 52).astype(np.float32)

    def create(z, z2=None, n=None, **cfg):
        g = sbt.Geometry(len(z) if n is None else n, z.ctypes.data, 5.1, 42.0,
                         z2.ctypes.data if z2 is not None else None)
        c = sbt.default_config(**cfg)
        h = ctypes.c_void_p()
        st = L.sbt_create(ctypes.byref(g), ctypes.byref(c), ctypes.byref(h))
        return st, L.sbt_last_error(None).decode()

    bad_z = mz.copy(); bad_z[7] = np.nan
    bad_z2 = mz.copy(); bad_z2[3] = np.inf
    cases = [
        (dict(z=mz, n=2), "n_modules"),
        (dict(z=mz, n=65), "n_modules"),
        (dict(z=bad_z), "finite"),
        (dict(z=mz, z2=bad_z2), "finite"),
        (dict(z=mz, k_doublets=0), "configuration"),
        (dict(z=mz, max_hits_per_event=16385), "configuration"),
        (dict(z=mz, threads_per_block=96), "configuration"),
        (dict(z=mz, gec_max_hits=-1), "configuration"),
        (dict(z=mz, hit_sigma=0.0), "configuration"),
    ]
    for kw, why in cases:
        st, msg = create(**kw)
        assert st == sbt.SBT_ERR_ARG and why in msg, (kw, st, msg)
    assert L.sbt_create(None, None, None) == sbt.SBT_ERR_ARG

"""CPU checks of the C ABI boundary: the library builds for sm_103a, loads,
and exports every entry point include/aleweno.h declares (no compute call
runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_1408_3719_gb300 import aleweno, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "aleweno.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(aw_[a-z0-9_]+)\s*\(", txt)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(aleweno.EXPORTED) == names


def test_invalid_config_is_rejected_without_gpu():
    lib = aleweno.load()
    cfg = aleweno.AwConfig(7, 1.4, 0.5, 20, 1.0, 0, 0, 0, None)
    h = ctypes.c_void_p()
    assert lib.aw_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    assert lib.aw_create(None, ctypes.byref(h)) == -1


def test_binding_fails_loudly_when_library_missing(tmp_path):
    import importlib
    mod = importlib.reload(aleweno)
    try:
        with pytest.raises(RuntimeError):
            mod._lib = None
            mod.load(str(tmp_path / "missing.so"))
    finally:
        importlib.reload(aleweno)

"""The C ABI library builds and exports every entry point include/cc.h declares (no GPU)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(cc_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    import paper_1908_11248_gb300 as cc

    return cc


def test_exports_every_declared_symbol(lib):
    names = declared()
    assert len(names) >= 20
    L = ctypes.CDLL(lib.LIB_PATH)
    for name in names:
        assert hasattr(L, name), name
    assert sorted(lib.EXPORTS) == names


def test_strerror_without_gpu(lib):
    assert lib.cc_strerror(0) == "ok"
    assert "capacity" in lib.cc_strerror(lib.CC_ECAPACITY)


def test_binding_fails_loudly_when_not_built(monkeypatch, lib):
    import paper_1908_11248_gb300 as cc

    monkeypatch.setattr(cc, "LIB_PATH", "/nonexistent/libcc.so")
    monkeypatch.setattr(cc, "_lib", None)
    with pytest.raises(RuntimeError):
        cc.lib()

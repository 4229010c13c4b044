"""The C-ABI library builds, loads and exports every entry point declared in
include/*.h (no compute call: this runs without a GPU)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in sorted(glob.glob(os.path.join(ROOT, "include", "*.h"))):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(pm_[a-z0-9_]+)\s*\(", text, re.M)
    return names


def test_headers_declare_entry_points():
    names = declared_symbols()
    assert "pm_polymul" in names and "pm_unpack" in names and "pm_strerror" in names


def test_library_exports_every_declared_symbol():
    from paper_1303_7425_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_declared_symbols():
    import paper_1303_7425_gb300 as P
    assert set(declared_symbols()) == set(P.SYMBOLS)


def test_strerror_and_version_without_gpu():
    import paper_1303_7425_gb300 as P
    L = P.lib()
    assert L.pm_strerror(0) == b"success"
    assert L.pm_strerror(-4).startswith(b"output capacity")
    assert L.pm_version() >= 100

"""The C-ABI libraries build, load and export every entry point declared in
include/*.h (no compute call: this runs without a GPU).  include/polymul.h is
the product's C-ABI (libpolymul.so); include/polymul_probe.h holds the
roofline's measurement probes (libpolymul_probe.so)."""

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_LIB = {"polymul.h": "libpolymul.so", "polymul_probe.h": "libpolymul_probe.so"}


def declared_symbols(header=None):
    names = []
    for h in sorted(HEADER_LIB) if header is None else [header]:
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(pm_[a-z0-9_]+)\s*\(", text, re.M)
    return names


def test_every_header_has_a_library():
    headers = sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h"))
    assert headers == sorted(HEADER_LIB)


def test_headers_declare_entry_points():
    names = declared_symbols("polymul.h")
    assert "pm_polymul" in names and "pm_unpack" in names and "pm_strerror" in names
    assert "pm_probe_oprate" in declared_symbols("polymul_probe.h")


def test_libraries_export_every_declared_symbol():
    from paper_1303_7425_gb300 import build as B
    B.build()
    for header, libname in HEADER_LIB.items():
        lib = ctypes.CDLL(os.path.join(ROOT, "paper_1303_7425_gb300", libname))
        missing = [n for n in declared_symbols(header) if not hasattr(lib, n)]
        assert not missing, (libname, missing)


def test_product_library_carries_no_probe():
    from paper_1303_7425_gb300 import build as B
    lib = ctypes.CDLL(B.build())
    assert not any(hasattr(lib, n) for n in declared_symbols("polymul_probe.h"))


def test_binding_lists_declared_symbols():
    import paper_1303_7425_gb300 as P
    assert set(declared_symbols("polymul.h")) == set(P.SYMBOLS)
    assert set(declared_symbols("polymul_probe.h")) == set(P.PROBE_SYMBOLS)


def test_strerror_and_version_without_gpu():
    import paper_1303_7425_gb300 as P
    L = P.lib()
    assert L.pm_strerror(0) == b"success"
    assert L.pm_strerror(-4).startswith(b"output capacity")
    assert L.pm_version() >= 100

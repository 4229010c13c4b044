"""Python access to the C oracle (oracle.c), and the exact-integer product
(exact.py) for the 192-bit kind.

TEST INFRASTRUCTURE ONLY: the tests, the package's smoke check and the
benchmark's CPU-baseline leg use this module; the library never does.  This
file only compiles oracle.c with gcc and marshals numpy arrays through ctypes.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional, Sequence, Tuple

import numpy as np

from .exact import ExactError, mul_exact, words192  # noqa: F401

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

OR_OK, OR_EINVAL, OR_EEXP_OVERFLOW, OR_ECOEF_BOUND, OR_ENOMEM = 0, -1, -2, -3, -5
KIND = {"m61": 0, "i64": 1, "i128": 2}


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle error {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain gcc, no GPU)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "oracle.h"))):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, SRC,
                               "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def build_variant(plant: int, out_path: str) -> str:
    """Compile oracle.c with a planted mistake (mutation tests only)."""
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", f"-DORACLE_PLANT={plant}",
                           "-o", out_path, SRC, "-lpthread"])
    return out_path


def lib():
    global _lib
    if _lib is None:
        _lib = _load(build())
    return _lib


def _load(path):
    L = C.CDLL(path)
    p, u32, u64, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int
    L.oracle_mul.argtypes = [u32, p, i32, p, p, u64, p, p, u64, p, p, p]
    L.oracle_mul.restype = i32
    L.oracle_mul_alg1.argtypes = [u32, p, i32, p, p, u64, p, p, u64, u32, u32, p, p, p, p]
    L.oracle_mul_alg1.restype = i32
    L.oracle_coef_at.argtypes = [u32, p, i32, p, p, u64, p, p, u64, p, u64, p]
    L.oracle_coef_at.restype = i32
    L.oracle_eval.argtypes = [u32, i32, p, p, u64, p]
    L.oracle_eval.restype = u64
    L.oracle_grid.argtypes = [p, u64, p, u64, u32, p, u64]
    L.oracle_grid.restype = u64
    L.oracle_free.argtypes = [p]
    L.oracle_free.restype = None
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a.size else None


def _prep(exps, coefs, kind):
    e = np.ascontiguousarray(exps, dtype=np.uint32)
    c = np.ascontiguousarray(coefs, dtype=np.uint64 if kind == "m61" else np.int64)
    return e, c


def _take(nv, kind, he, hc, nh):
    n = int(nh.value)
    L = lib()
    if n:
        e = np.ctypeslib.as_array(C.cast(he, C.POINTER(C.c_uint32)), shape=(n * nv,)).copy().reshape(n, nv)
        words = n if kind == "m61" else 2 * n
        c = np.ctypeslib.as_array(C.cast(hc, C.POINTER(C.c_uint64)), shape=(words,)).copy()
        if kind != "m61":
            c = c.reshape(n, 2)
    else:
        e = np.zeros((0, nv), dtype=np.uint32)
        c = np.zeros((0,) if kind == "m61" else (0, 2), dtype=np.uint64)
    L.oracle_free(he)
    L.oracle_free(hc)
    return e, c


def mul(nvars: int, field_bits: Sequence[int], kind: str, fe, fc, ge, gc) -> Tuple[np.ndarray, np.ndarray]:
    """Full product by the definition.  Returns (exps (n, nvars) uint32,
    coefs): uint64 residues for kind 'm61', (n, 2) uint64 (lo, hi) int128
    words for kind 'i64'.  Raises OracleError on the error rules."""
    fe, fc = _prep(fe, fc, kind)
    ge, gc = _prep(ge, gc, kind)
    w = np.ascontiguousarray(field_bits, dtype=np.uint8)
    he, hc, nh = C.c_void_p(), C.c_void_p(), C.c_uint64()
    rc = lib().oracle_mul(nvars, _ptr(w), KIND[kind], _ptr(fe), _ptr(fc), fe.shape[0],
                          _ptr(ge), _ptr(gc), ge.shape[0], C.byref(he), C.byref(hc), C.byref(nh))
    if rc != OR_OK:
        raise OracleError(rc)
    return _take(nvars, kind, he, hc, nh)


def mul_alg1(nvars: int, field_bits: Sequence[int], kind: str, fe, fc, ge, gc,
             l: int = 64, threads: int = 1) -> Tuple[np.ndarray, np.ndarray, int]:
    """Alg. 1 of the paper on CPU threads; returns (exps, coefs, n_intervals)."""
    fe, fc = _prep(fe, fc, kind)
    ge, gc = _prep(ge, gc, kind)
    w = np.ascontiguousarray(field_bits, dtype=np.uint8)
    he, hc, nh, ni = C.c_void_p(), C.c_void_p(), C.c_uint64(), C.c_uint64()
    rc = lib().oracle_mul_alg1(nvars, _ptr(w), KIND[kind], _ptr(fe), _ptr(fc), fe.shape[0],
                               _ptr(ge), _ptr(gc), ge.shape[0], l, threads,
                               C.byref(he), C.byref(hc), C.byref(nh), C.byref(ni))
    if rc != OR_OK:
        raise OracleError(rc)
    e, c = _take(nvars, kind, he, hc, nh)
    return e, c, int(ni.value)


def coef_at(nvars: int, field_bits: Sequence[int], kind: str, fe, fc, ge, gc, gammas) -> np.ndarray:
    """Coefficient of each monomial in gammas (k, nvars) in the product."""
    fe, fc = _prep(fe, fc, kind)
    ge, gc = _prep(ge, gc, kind)
    w = np.ascontiguousarray(field_bits, dtype=np.uint8)
    gm = np.ascontiguousarray(gammas, dtype=np.uint32).reshape(-1, nvars)
    k = gm.shape[0]
    out = np.zeros(k if kind == "m61" else (k, 2), dtype=np.uint64)
    rc = lib().oracle_coef_at(nvars, _ptr(w), KIND[kind], _ptr(fe), _ptr(fc), fe.shape[0],
                              _ptr(ge), _ptr(gc), ge.shape[0], _ptr(gm), k, _ptr(out))
    if rc != OR_OK:
        raise OracleError(rc)
    return out


def evaluate(nvars: int, kind: str, exps, coefs, r: Sequence[int]) -> int:
    """p(r) mod 2^61-1; kind 'm61' (uint64), 'i64' (int64) or 'i128' ((n,2) words)."""
    e = np.ascontiguousarray(exps, dtype=np.uint32).reshape(-1, nvars)
    if kind == "m61":
        c = np.ascontiguousarray(coefs, dtype=np.uint64)
    elif kind == "i64":
        c = np.ascontiguousarray(coefs, dtype=np.int64)
    else:
        c = np.ascontiguousarray(coefs, dtype=np.uint64).reshape(-1, 2)
    rr = np.ascontiguousarray([int(x) for x in r], dtype=np.uint64)
    return int(lib().oracle_eval(nvars, KIND[kind], _ptr(e), _ptr(c), e.shape[0], _ptr(rr)))


def grid(alpha: np.ndarray, beta: np.ndarray, l: int) -> np.ndarray:
    """The Sec. 5 grid S* (unsorted, without gamma_end) for sorted packed keys."""
    a = np.ascontiguousarray(alpha, dtype=np.uint64)
    b = np.ascontiguousarray(beta, dtype=np.uint64)
    L = lib()
    n = int(L.oracle_grid(_ptr(a), a.size, _ptr(b), b.size, l, None, 0))
    out = np.zeros(n, dtype=np.uint64)
    L.oracle_grid(_ptr(a), a.size, _ptr(b), b.size, l, _ptr(out), n)
    return out


def i128_to_int(words: np.ndarray) -> list:
    """(n, 2) uint64 (lo, hi) words -> Python ints (two's complement)."""
    out = []
    for lo, hi in np.asarray(words, dtype=np.uint64).reshape(-1, 2):
        v = (int(hi) << 64) | int(lo)
        out.append(v - (1 << 128) if v >> 127 else v)
    return out

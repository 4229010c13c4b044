"""ctypes binding of libpolymul.so (include/polymul.h).

Argument marshalling only: tensors are passed to the C-ABI as raw device
pointers with the current CUDA stream; every step of the product runs in the
library's kernels.  There is no fallback: if the library is missing or no
CUDA device is present the calls raise.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpolymul.so")

PM_MAX_VARS = 16
PM_OK, PM_EINVAL, PM_EEXP_OVERFLOW, PM_ECOEF_BOUND = 0, -1, -2, -3
PM_ECAPACITY, PM_ENOMEM, PM_ETIMEOUT, PM_ECUDA, PM_EPLAN, PM_ECANCELED = -4, -5, -6, -7, -8, -9
KIND = {"m61": 0, "i64": 1, "i192": 2}
STRATEGY = {"auto": 0, "direct": 1, "sort": 2, "hash": 3, "bucket": 4}
STRATEGY_NAME = {v: k for k, v in STRATEGY.items()}
ACCUMULATOR = {"auto": 0, "wide": 1, "limbs": 2, "limbs3": 3}


class pm_packing(C.Structure):
    _fields_ = [("nvars", C.c_uint32), ("field_bits", C.c_uint8 * PM_MAX_VARS)]


class pm_terms_in(C.Structure):
    _fields_ = [("exps", C.c_void_p), ("coefs", C.c_void_p), ("n", C.c_uint64)]


class pm_terms_out(C.Structure):
    _fields_ = [("keys", C.c_void_p), ("coefs", C.c_void_p), ("n", C.c_uint64), ("cap", C.c_uint64)]


class pm_options(C.Structure):
    _fields_ = [("strategy", C.c_int32), ("slots", C.c_uint32), ("chunk", C.c_uint32),
                ("ranges_per_sm", C.c_uint32), ("accumulator", C.c_int32), ("cost_row", C.c_uint32),
                ("cost_window", C.c_uint32), ("grid_l", C.c_uint32)]


class pm_stats(C.Structure):
    _fields_ = [("n_f", C.c_uint64), ("n_g", C.c_uint64), ("term_products", C.c_uint64),
                ("n_out", C.c_uint64), ("n_ranges", C.c_uint64), ("box", C.c_uint64),
                ("strategy", C.c_int32), ("refine_rounds", C.c_uint32),
                ("kernel_launches", C.c_uint32), ("host_syncs", C.c_uint32),
                ("ms_range_kernel", C.c_float), ("ms_range_step", C.c_float)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["strategy"] = STRATEGY_NAME.get(d["strategy"], d["strategy"])
        return d


class PolymulError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        msg = lib().pm_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")
        self.code = code


# exported symbols, in include/polymul.h order
SYMBOLS = ("pm_polymul", "pm_workspace_size", "pm_polymul_ws", "pm_shard_bounds", "pm_polymul_range",
           "pm_split_cumulative", "pm_out_bound", "pm_grid", "pm_unpack", "pm_pack", "pm_autotune", "pm_batch_autotune",
           "pm_batch_plan_create", "pm_batch_plan_run",
           "pm_batch_plan_finish", "pm_batch_plan_destroy", "pm_batch_polymul", "pm_batch_workspace",
           "pm_batch_enqueue", "pm_batch_collect", "pm_server_create", "pm_server_submit", "pm_server_cancel", "pm_server_progress",
           "pm_server_state", "pm_server_destroy", "pm_polymul_noalloc",
           "pm_plan_create", "pm_plan_run", "pm_plan_finish", "pm_plan_finish_to_host", "pm_plan_captured",
           "pm_plan_destroy",
           "pm_strerror", "pm_version")
# exported by libpolymul_probe.so, in include/polymul_probe.h order
PROBE_SYMBOLS = ("pm_probe_mac", "pm_probe_oprate", "pm_probe_ops_per_step")
PROBE_LIB_PATH = os.path.join(HERE, "libpolymul_probe.so")
OP = {"imad_wide": 0, "imad": 1, "iadd3": 2, "lop3": 3, "shf": 4, "imad_hi": 6}

_lib = None


def lib():
    """Load libpolymul.so (no compute call is made here)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_1303_7425_gb300.build.build() first")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER
        L.pm_polymul.argtypes = [P(pm_packing), C.c_int, P(pm_terms_in), P(pm_terms_in), P(pm_terms_out),
                                 P(pm_options), P(pm_stats), C.c_void_p]
        L.pm_polymul.restype = C.c_int
        L.pm_workspace_size.argtypes = [P(pm_packing), C.c_int, P(pm_terms_in), P(pm_terms_in), P(pm_options),
                                        P(C.c_uint64), P(C.c_uint64), C.c_void_p]
        L.pm_workspace_size.restype = C.c_int
        L.pm_polymul_ws.argtypes = [P(pm_packing), C.c_int, P(pm_terms_in), P(pm_terms_in), P(pm_terms_out),
                                    P(pm_options), P(pm_stats), C.c_void_p, C.c_uint64, C.c_void_p]
        L.pm_polymul_ws.restype = C.c_int
        L.pm_out_bound.argtypes = [P(pm_packing), P(pm_terms_in), P(pm_terms_in), P(C.c_uint64), C.c_void_p]
        L.pm_out_bound.restype = C.c_int
        L.pm_shard_bounds.argtypes = [P(pm_packing), C.c_int, P(pm_terms_in), P(pm_terms_in), C.c_uint32,
                                      C.c_void_p, C.c_void_p, C.c_void_p]
        L.pm_shard_bounds.restype = C.c_int
        L.pm_polymul_range.argtypes = [P(pm_packing), C.c_int, P(pm_terms_in), P(pm_terms_in), C.c_uint64,
                                       C.c_uint64, P(pm_terms_out), P(pm_options), P(pm_stats), C.c_void_p]
        L.pm_polymul_range.restype = C.c_int
        L.pm_split_cumulative.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, C.c_void_p]
        L.pm_split_cumulative.restype = C.c_int
        L.pm_grid.argtypes = [C.c_void_p, C.c_uint64, C.c_void_p, C.c_uint64, C.c_uint32, C.c_void_p, C.c_uint64,
                              P(C.c_uint64), C.c_void_p]
        L.pm_grid.restype = C.c_int
        L.pm_unpack.argtypes = [P(pm_packing), C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]
        L.pm_unpack.restype = C.c_int
        L.pm_pack.argtypes = [P(pm_packing), C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]
        L.pm_pack.restype = C.c_int
        L.pm_polymul_noalloc.argtypes = [P(pm_packing), C.c_int, P(pm_terms_in), P(pm_terms_in),
                                         P(pm_terms_out), C.c_void_p]
        L.pm_polymul_noalloc.restype = C.c_int
        L.pm_strerror.argtypes = [C.c_int]
        L.pm_strerror.restype = C.c_char_p
        L.pm_version.argtypes = []
        L.pm_version.restype = C.c_int
        _lib = L
    return _lib


def packing(field_bits: Sequence[int]) -> pm_packing:
    pk = pm_packing()
    pk.nvars = len(field_bits)
    for v, w in enumerate(field_bits[:PM_MAX_VARS]):
        pk.field_bits[v] = int(w)
    return pk


def options(strategy: str = "auto", slots: int = 0, chunk: int = 0, ranges_per_sm: int = 0,
            accumulator: str = "auto", cost_row: int = 0, cost_window: int = 0, grid_l: int = 0) -> pm_options:
    o = pm_options()
    o.strategy = STRATEGY[strategy]
    o.slots = slots
    o.chunk = chunk
    o.ranges_per_sm = ranges_per_sm
    o.accumulator = ACCUMULATOR[accumulator]
    o.cost_row = cost_row
    o.cost_window = cost_window
    o.grid_l = grid_l
    return o


def _stream_handle(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _terms_in(exps, coefs) -> pm_terms_in:
    t = pm_terms_in()
    n = int(exps.shape[0])
    t.n = n
    t.exps = exps.data_ptr() if n else None
    t.coefs = coefs.data_ptr() if n else None
    return t


def _check_cuda(*tensors):
    import torch
    dev = None
    for x in tensors:
        if not x.is_cuda:
            raise ValueError("inputs must be CUDA tensors")
        if not x.is_contiguous():
            raise ValueError("inputs must be contiguous")
        if dev is None:
            dev = torch.cuda.current_device()
        if x.device.index != dev:
            raise ValueError(f"tensor on cuda:{x.device.index}, but the current device is cuda:{dev}")


WORDS = {"m61": 1, "i64": 2, "i192": 3}


def _dtype_names(t) -> str:
    return str(t.dtype).replace("torch.", "")


def check_operands(field_bits, f_exps, f_coefs, g_exps, g_coefs, kind: str = "m61") -> None:
    """Shapes and element types of two operands, checked before any pointer
    reaches the library: exps (n, nvars) 32-bit integers, coefs (n,) 64-bit
    integers.  Raises ValueError.  Works on tensors of any device."""
    if kind not in WORDS:
        raise ValueError(f"unknown coefficient kind {kind!r}")
    nv = len(field_bits)
    for name, e, c in (("f", f_exps, f_coefs), ("g", g_exps, g_coefs)):
        if e.dim() != 2 or int(e.shape[1]) != nv:
            raise ValueError(f"{name}_exps must have shape (n, {nv}), got {tuple(e.shape)}")
        if _dtype_names(e) not in ("int32", "uint32"):
            raise ValueError(f"{name}_exps must hold 32-bit integers, got {e.dtype}")
        if c.dim() != 1 or int(c.shape[0]) != int(e.shape[0]):
            raise ValueError(f"{name}_coefs must have shape ({int(e.shape[0])},), got {tuple(c.shape)}")
        if _dtype_names(c) not in ("int64", "uint64"):
            raise ValueError(f"{name}_coefs must hold 64-bit integers, got {c.dtype}")


def check_out(out, kind: str = "m61") -> int:
    """The caller's output pair (keys (cap,), coefs (cap,) for m61 or
    (cap, words) for the wider kinds), 64-bit integers; returns cap.
    Raises ValueError.  Works on tensors of any device."""
    if kind not in WORDS:
        raise ValueError(f"unknown coefficient kind {kind!r}")
    keys, coefs = out
    if keys.dim() != 1 or _dtype_names(keys) not in ("int64", "uint64"):
        raise ValueError(f"output keys must be a (cap,) tensor of 64-bit integers, got {tuple(keys.shape)} "
                         f"{keys.dtype}")
    cap = int(keys.shape[0])
    words = WORDS[kind]
    want = (cap,) if words == 1 else (cap, words)
    if tuple(int(x) for x in coefs.shape) != want or _dtype_names(coefs) not in ("int64", "uint64"):
        raise ValueError(f"output coefs for kind {kind!r} must be a {want} tensor of 64-bit integers, got "
                         f"{tuple(coefs.shape)} {coefs.dtype}")
    return cap


@dataclass
class Product:
    keys: "object"            # (n,) int64 tensor holding uint64 packed keys
    coefs: "object"           # (n,) int64 residues, or (n, 2) int128 / (n, 3) int192 words, low word first
    n: int
    stats: dict


def out_bound(field_bits, f_exps, g_exps, stream=None) -> int:
    _check_cuda(f_exps, g_exps)
    pk = packing(field_bits)
    f = _terms_in(f_exps, f_exps)
    g = _terms_in(g_exps, g_exps)
    b = C.c_uint64(0)
    rc = lib().pm_out_bound(C.byref(pk), C.byref(f), C.byref(g), C.byref(b), _stream_handle(stream))
    if rc != PM_OK:
        raise PolymulError(rc, "pm_out_bound")
    return int(b.value)


def polymul(field_bits: Sequence[int], f_exps, f_coefs, g_exps, g_coefs, kind: str = "m61",
            strategy: str = "auto", slots: int = 0, chunk: int = 0, ranges_per_sm: int = 0,
            accumulator: str = "auto", out=None, stream=None, cost_row: int = 0, cost_window: int = 0,
            grid_l: int = 0) -> Product:
    """h = f * g on the current CUDA device.

    f_exps/g_exps: (n, nvars) int32/uint32 CUDA tensors; f_coefs/g_coefs: (n,)
    int64/uint64 CUDA tensors.  ``out``: optional (keys, coefs) tensors to
    write into (their length is the capacity); otherwise they are allocated
    from pm_out_bound."""
    import torch
    check_operands(field_bits, f_exps, f_coefs, g_exps, g_coefs, kind)
    if out is not None:
        check_out(out, kind)
        _check_cuda(out[0], out[1])
    _check_cuda(f_exps, f_coefs, g_exps, g_coefs)
    words = WORDS[kind]
    pk = packing(field_bits)
    f = _terms_in(f_exps, f_coefs)
    g = _terms_in(g_exps, g_coefs)
    if out is None:
        cap = out_bound(field_bits, f_exps, g_exps, stream)
        keys = torch.empty(max(cap, 1), dtype=torch.int64, device=f_exps.device)
        coefs = torch.empty((max(cap, 1), words) if words > 1 else (max(cap, 1),), dtype=torch.int64,
                            device=f_exps.device)
    else:
        keys, coefs = out
        cap = int(keys.shape[0])
    h = pm_terms_out()
    h.keys = keys.data_ptr()
    h.coefs = coefs.data_ptr()
    h.cap = cap
    st = pm_stats()
    o = options(strategy, slots, chunk, ranges_per_sm, accumulator, cost_row, cost_window, grid_l)
    rc = lib().pm_polymul(C.byref(pk), KIND[kind], C.byref(f), C.byref(g), C.byref(h), C.byref(o),
                          C.byref(st), _stream_handle(stream))
    if rc != PM_OK:
        err = PolymulError(rc, "pm_polymul")
        err.needed = int(h.n)
        raise err
    n = int(h.n)
    return Product(keys[:n], coefs[:n], n, st.as_dict())


def shard_bounds(field_bits: Sequence[int], f_exps, f_coefs, g_exps, g_coefs, nshards: int, kind: str = "m61",
                 stream=None):
    """Alg. 2's split of the output key space into ``nshards`` slices of
    about equal term-product counts (pm_shard_bounds).  Returns (bounds: list
    of nshards + 1 ints, products: list of nshards ints)."""
    import numpy as np
    check_operands(field_bits, f_exps, f_coefs, g_exps, g_coefs, kind)
    _check_cuda(f_exps, f_coefs, g_exps, g_coefs)
    pk = packing(field_bits)
    f = _terms_in(f_exps, f_coefs)
    g = _terms_in(g_exps, g_coefs)
    bounds = np.zeros(nshards + 1, dtype=np.uint64)
    prods = np.zeros(nshards, dtype=np.uint64)
    rc = lib().pm_shard_bounds(C.byref(pk), KIND[kind], C.byref(f), C.byref(g), nshards,
                               bounds.ctypes.data_as(C.c_void_p), prods.ctypes.data_as(C.c_void_p),
                               _stream_handle(stream))
    if rc != PM_OK:
        raise PolymulError(rc, "pm_shard_bounds")
    return [int(x) for x in bounds], [int(x) for x in prods]


def polymul_range(field_bits: Sequence[int], f_exps, f_coefs, g_exps, g_coefs, key_lo: int, key_hi: int,
                  kind: str = "m61", out=None, stream=None, strategy: str = "auto", **opts) -> Product:
    """The result terms of f * g whose packed key lies in [key_lo, key_hi)
    (pm_polymul_range).  ``out``: optional (keys, coefs); otherwise sized
    by pm_out_bound."""
    import torch
    check_operands(field_bits, f_exps, f_coefs, g_exps, g_coefs, kind)
    if out is not None:
        check_out(out, kind)
        _check_cuda(out[0], out[1])
    _check_cuda(f_exps, f_coefs, g_exps, g_coefs)
    words = WORDS[kind]
    pk = packing(field_bits)
    f = _terms_in(f_exps, f_coefs)
    g = _terms_in(g_exps, g_coefs)
    if out is None:
        cap = out_bound(field_bits, f_exps, g_exps, stream)
        keys = torch.empty(max(cap, 1), dtype=torch.int64, device=f_exps.device)
        coefs = torch.empty((max(cap, 1), words) if words > 1 else (max(cap, 1),), dtype=torch.int64,
                            device=f_exps.device)
    else:
        keys, coefs = out
        cap = int(keys.shape[0])
    h = pm_terms_out(keys.data_ptr(), coefs.data_ptr(), 0, cap)
    st = pm_stats()
    o = options(strategy, **opts)
    rc = lib().pm_polymul_range(C.byref(pk), KIND[kind], C.byref(f), C.byref(g), int(key_lo) & (2**64 - 1),
                                int(key_hi) & (2**64 - 1), C.byref(h), C.byref(o), C.byref(st),
                                _stream_handle(stream))
    if rc != PM_OK:
        err = PolymulError(rc, "pm_polymul_range")
        err.needed = int(h.n)
        raise err
    n = int(h.n)
    return Product(keys[:n], coefs[:n], n, st.as_dict())


def split_cumulative(cum, nshards: int):
    """pm_split_cumulative on host arrays (no GPU): the interval boundary
    index each of ``nshards`` shards starts at, for ascending cumulative
    operation counts ``cum``.  Returns nshards + 1 ints."""
    import numpy as np
    c = np.ascontiguousarray(cum, dtype=np.uint64)
    cut = np.zeros(nshards + 1, dtype=np.uint32)
    rc = lib().pm_split_cumulative(c.ctypes.data_as(C.c_void_p), c.size, nshards, cut.ctypes.data_as(C.c_void_p))
    if rc != PM_OK:
        raise PolymulError(rc, "pm_split_cumulative")
    return [int(x) for x in cut]


def workspace_size(field_bits: Sequence[int], f_exps, f_coefs, g_exps, g_coefs, kind: str = "m61",
                   strategy: str = "auto", stream=None, **opts):
    """(workspace bytes, result terms) of the product on these inputs
    (pm_workspace_size: the product runs once, nothing is written)."""
    check_operands(field_bits, f_exps, f_coefs, g_exps, g_coefs, kind)
    _check_cuda(f_exps, f_coefs, g_exps, g_coefs)
    pk = packing(field_bits)
    f = _terms_in(f_exps, f_coefs)
    g = _terms_in(g_exps, g_coefs)
    o = options(strategy, **opts)
    ws, n = C.c_uint64(0), C.c_uint64(0)
    rc = lib().pm_workspace_size(C.byref(pk), KIND[kind], C.byref(f), C.byref(g), C.byref(o), C.byref(ws),
                                 C.byref(n), _stream_handle(stream))
    if rc != PM_OK:
        raise PolymulError(rc, "pm_workspace_size")
    return int(ws.value), int(n.value)


def polymul_ws(field_bits: Sequence[int], f_exps, f_coefs, g_exps, g_coefs, out, workspace,
               kind: str = "m61", strategy: str = "auto", stream=None, **opts) -> Product:
    """h = f * g with all scratch carved from ``workspace`` (a CUDA uint8
    tensor, 256-byte aligned, sized by workspace_size): the call allocates
    no device memory.  ``out`` = (keys, coefs) supplied by the caller."""
    check_operands(field_bits, f_exps, f_coefs, g_exps, g_coefs, kind)
    cap = check_out(out, kind)
    _check_cuda(f_exps, f_coefs, g_exps, g_coefs, out[0], out[1], workspace)
    pk = packing(field_bits)
    f = _terms_in(f_exps, f_coefs)
    g = _terms_in(g_exps, g_coefs)
    h = pm_terms_out()
    h.keys = out[0].data_ptr()
    h.coefs = out[1].data_ptr()
    h.cap = cap
    st = pm_stats()
    o = options(strategy, **opts)
    nbytes = int(workspace.numel()) * int(workspace.element_size())
    rc = lib().pm_polymul_ws(C.byref(pk), KIND[kind], C.byref(f), C.byref(g), C.byref(h), C.byref(o),
                             C.byref(st), workspace.data_ptr() if nbytes else None, nbytes, _stream_handle(stream))
    if rc != PM_OK:
        err = PolymulError(rc, "pm_polymul_ws")
        err.needed = int(h.n)
        raise err
    n = int(h.n)
    return Product(out[0][:n], out[1][:n], n, st.as_dict())


def _plan_lib():
    L = lib()
    if not getattr(L, "_plan_ready", False):
        P = C.POINTER
        L.pm_plan_create.argtypes = [P(pm_packing), C.c_int, P(pm_terms_in), P(pm_terms_in), P(pm_terms_out),
                                     P(pm_options), P(C.c_void_p), C.c_void_p]
        L.pm_plan_create.restype = C.c_int
        L.pm_plan_run.argtypes = [C.c_void_p, C.c_void_p]
        L.pm_plan_run.restype = C.c_int
        L.pm_plan_finish.argtypes = [C.c_void_p, P(C.c_uint64), C.c_void_p]
        L.pm_plan_finish.restype = C.c_int
        L.pm_plan_finish_to_host.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, P(C.c_uint64),
                                             C.c_void_p]
        L.pm_plan_finish_to_host.restype = C.c_int
        L.pm_plan_captured.argtypes = [C.c_void_p]
        L.pm_plan_captured.restype = C.c_int
        L.pm_plan_destroy.argtypes = [C.c_void_p]
        L.pm_plan_destroy.restype = None
        L._plan_ready = True
    return L


class Plan:
    """One product, repeated: pm_plan_* (a CUDA graph of the whole device path).

    Creating the plan computes the product once into ``out`` (keys, coefs
    tensors; their length is the capacity).  ``run()`` enqueues a replay on
    the current contents of the input tensors, ``finish()`` waits and returns
    the result size (raises PolymulError with PM_EPLAN when the inputs no
    longer match the plan).  The tensors must stay alive and unmoved while
    the plan exists."""

    def __init__(self, field_bits, f_exps, f_coefs, g_exps, g_coefs, out, kind: str = "m61",
                 strategy: str = "auto", slots: int = 0, chunk: int = 0, ranges_per_sm: int = 0,
                 accumulator: str = "auto", stream=None):
        check_operands(field_bits, f_exps, f_coefs, g_exps, g_coefs, kind)
        check_out(out, kind)
        _check_cuda(f_exps, f_coefs, g_exps, g_coefs, out[0], out[1])
        self._keep = (f_exps, f_coefs, g_exps, g_coefs, out)
        self.pk = packing(field_bits)
        self.f = _terms_in(f_exps, f_coefs)
        self.g = _terms_in(g_exps, g_coefs)
        self.h = pm_terms_out()
        self.h.keys = out[0].data_ptr()
        self.h.coefs = out[1].data_ptr()
        self.h.cap = int(out[0].shape[0])
        self.o = options(strategy, slots, chunk, ranges_per_sm, accumulator)
        self.handle = C.c_void_p()
        L = _plan_lib()
        rc = L.pm_plan_create(C.byref(self.pk), KIND[kind], C.byref(self.f), C.byref(self.g), C.byref(self.h),
                              C.byref(self.o), C.byref(self.handle), _stream_handle(stream))
        if rc != PM_OK:
            raise PolymulError(rc, "pm_plan_create")
        self.n = int(self.h.n)
        self.captured = bool(L.pm_plan_captured(self.handle))

    def run(self, stream=None):
        rc = _plan_lib().pm_plan_run(self.handle, _stream_handle(stream))
        if rc != PM_OK:
            raise PolymulError(rc, "pm_plan_run")

    def finish(self, stream=None) -> int:
        n = C.c_uint64(0)
        rc = _plan_lib().pm_plan_finish(self.handle, C.byref(n), _stream_handle(stream))
        if rc != PM_OK:
            err = PolymulError(rc, "pm_plan_finish")
            err.needed = int(n.value)
            raise err
        return int(n.value)

    def finish_to_host(self, host_keys, host_coefs, stream=None) -> int:
        """finish(), with the result also copied on the device side into the
        page-locked CPU tensors host_keys (cap,) and host_coefs (cap,) or
        (cap, words) (torch ``pin_memory()``): one host wait per product.
        Returns the result size."""
        for t in (host_keys, host_coefs):
            if t.is_cuda or not t.is_pinned() or not t.is_contiguous():
                raise PolymulError(PM_EINVAL, "host buffers must be contiguous page-locked CPU tensors")
        n = C.c_uint64(0)
        rc = _plan_lib().pm_plan_finish_to_host(self.handle, host_keys.data_ptr(), host_coefs.data_ptr(),
                                                int(host_keys.shape[0]), C.byref(n), _stream_handle(stream))
        if rc != PM_OK:
            err = PolymulError(rc, "pm_plan_finish_to_host")
            err.needed = int(n.value)
            raise err
        return int(n.value)

    def close(self):
        if self.handle:
            _plan_lib().pm_plan_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grid(alpha, beta, l: int, stream=None):
    """Step 1 of Alg. 1 (pm_grid): the Sec. 5 grid's splitters plus
    gamma_end, sorted and deduplicated, for ascending (n,) int64 tensors of
    packed keys.  Returns an int64 tensor holding the uint64 splitters."""
    import torch
    _check_cuda(alpha, beta)
    for t in (alpha, beta):
        if t.dim() != 1 or _dtype_names(t) not in ("int64", "uint64"):
            raise ValueError("keys must be (n,) tensors of 64-bit integers")
    na, nb = int(alpha.shape[0]), int(beta.shape[0])
    n = C.c_uint64(0)
    L = lib()
    rc = L.pm_grid(alpha.data_ptr() if na else None, na, beta.data_ptr() if nb else None, nb, l, None, 0,
                   C.byref(n), _stream_handle(stream))
    if rc not in (PM_OK, PM_ECAPACITY):
        raise PolymulError(rc, "pm_grid")
    out = torch.empty(max(int(n.value), 1), dtype=torch.int64, device=alpha.device)
    rc = L.pm_grid(alpha.data_ptr() if na else None, na, beta.data_ptr() if nb else None, nb, l, out.data_ptr(),
                   int(out.shape[0]), C.byref(n), _stream_handle(stream))
    if rc != PM_OK:
        raise PolymulError(rc, "pm_grid")
    return out[:int(n.value)]


def unpack(field_bits: Sequence[int], keys, stream=None):
    """(n,) packed keys -> (n, nvars) int32 exponent tensor."""
    import torch
    _check_cuda(keys)
    n = int(keys.shape[0])
    exps = torch.empty((n, len(field_bits)), dtype=torch.int32, device=keys.device)
    if n:
        rc = lib().pm_unpack(C.byref(packing(field_bits)), keys.data_ptr(), n, exps.data_ptr(),
                             _stream_handle(stream))
        if rc != PM_OK:
            raise PolymulError(rc, "pm_unpack")
    return exps


def pack(field_bits: Sequence[int], exps, stream=None):
    import torch
    _check_cuda(exps)
    n = int(exps.shape[0])
    keys = torch.empty(max(n, 1), dtype=torch.int64, device=exps.device)
    if n:
        rc = lib().pm_pack(C.byref(packing(field_bits)), exps.data_ptr(), n, keys.data_ptr(),
                           _stream_handle(stream))
        if rc != PM_OK:
            raise PolymulError(rc, "pm_pack")
    return keys[:n]


_probe_lib = None


def probe_lib():
    """Load libpolymul_probe.so, the roofline's measurement probes (a
    library of their own, not part of the product's C-ABI)."""
    global _probe_lib
    if _probe_lib is None:
        if not os.path.exists(PROBE_LIB_PATH):
            raise RuntimeError(f"{PROBE_LIB_PATH} is missing: run paper_1303_7425_gb300.build.build() first")
        L = C.CDLL(PROBE_LIB_PATH)
        L.pm_probe_mac.argtypes = [C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint64, C.c_void_p, C.c_void_p]
        L.pm_probe_mac.restype = C.c_int
        L.pm_probe_oprate.argtypes = [C.c_int, C.c_uint32, C.c_uint32, C.c_uint64, C.c_uint32, C.c_void_p,
                                      C.c_void_p, C.c_void_p]
        L.pm_probe_oprate.restype = C.c_int
        L.pm_probe_ops_per_step.argtypes = [C.c_int]
        L.pm_probe_ops_per_step.restype = C.c_uint32
        _probe_lib = L
    return _probe_lib


def probe_mac(blocks: int, threads: int, iters: int, sink, seed: int = 0x1303742500, stream=None) -> None:
    """Launch the register-only multiply-accumulate probe (see
    include/polymul_probe.h); time it with CUDA events on ``stream``."""
    _check_cuda(sink)
    rc = probe_lib().pm_probe_mac(blocks, threads, iters, seed, sink.data_ptr(), _stream_handle(stream))
    if rc != PM_OK:
        raise PolymulError(rc, "pm_probe_mac")


def probe_oprate(op: str, blocks: int, threads: int, iters: int, sink, clk=None, seed: int = 0x13037425,
                 stream=None) -> int:
    """Launch the op-rate probe of instruction class ``op`` (a key of OP);
    ``clk``: optional (2,) int64 CUDA tensor for the first block's SM cycles
    and nanoseconds.  Returns the instructions one thread issues per step."""
    _check_cuda(sink)
    if clk is not None:
        _check_cuda(clk)
    L = probe_lib()
    rc = L.pm_probe_oprate(OP[op], blocks, threads, iters, seed & 0xFFFFFFFF, sink.data_ptr(),
                           clk.data_ptr() if clk is not None else None, _stream_handle(stream))
    if rc != PM_OK:
        raise PolymulError(rc, "pm_probe_oprate")
    return int(L.pm_probe_ops_per_step(OP[op]))


NOALLOC_MAX_TERMS = 4096
NOALLOC_MAX_PRODUCTS = 65536


def polymul_noalloc(field_bits: Sequence[int], f_exps, f_coefs, g_exps, g_coefs, out, kind: str = "m61",
                    stream=None) -> int:
    """The product through pm_polymul_noalloc, for callers that cannot
    allocate device memory: the library allocates nothing (its scratch is a
    static device array); ``out`` = (keys, coefs) tensors supplied by the
    caller.  Returns the number of result terms written."""
    check_operands(field_bits, f_exps, f_coefs, g_exps, g_coefs, kind)
    check_out(out, kind)
    _check_cuda(f_exps, f_coefs, g_exps, g_coefs, out[0], out[1])
    pk = packing(field_bits)
    f = _terms_in(f_exps, f_coefs)
    g = _terms_in(g_exps, g_coefs)
    h = pm_terms_out()
    h.keys = out[0].data_ptr()
    h.coefs = out[1].data_ptr()
    h.cap = int(out[0].shape[0])
    rc = lib().pm_polymul_noalloc(C.byref(pk), KIND[kind], C.byref(f), C.byref(g), C.byref(h),
                                  _stream_handle(stream))
    if rc != PM_OK:
        err = PolymulError(rc, "pm_polymul_noalloc")
        err.needed = int(h.n)
        raise err
    return int(h.n)


# ---------------------------------------------------------------------------
# batches (pm_batch_*)
# ---------------------------------------------------------------------------

BATCH_MAX_TERMS = 8192


class pm_batch_item(C.Structure):
    _fields_ = [("pk", pm_packing), ("coef_kind", C.c_int32), ("f", pm_terms_in), ("g", pm_terms_in),
                ("h", pm_terms_out), ("status", C.c_int32)]


class pm_batch_options(C.Structure):
    _fields_ = [("range_target", C.c_uint32), ("ranges_per_item", C.c_uint32)]


class pm_batch_stats(C.Structure):
    _fields_ = [("term_products", C.c_uint64), ("n_out", C.c_uint64), ("n_ranges", C.c_uint64),
                ("work_items", C.c_uint64), ("kernel_launches", C.c_uint32), ("graph", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_batch_ready = False


def _batch_lib():
    global _batch_ready
    L = lib()
    if not _batch_ready:
        P = C.POINTER
        L.pm_batch_plan_create.argtypes = [P(pm_batch_item), C.c_uint32, P(pm_batch_options), P(C.c_void_p),
                                           C.c_void_p]
        L.pm_batch_plan_create.restype = C.c_int
        L.pm_batch_plan_run.argtypes = [C.c_void_p, C.c_void_p]
        L.pm_batch_plan_run.restype = C.c_int
        L.pm_batch_plan_finish.argtypes = [C.c_void_p, P(pm_batch_item), P(pm_batch_stats), C.c_void_p]
        L.pm_batch_plan_finish.restype = C.c_int
        L.pm_batch_plan_destroy.argtypes = [C.c_void_p]
        L.pm_batch_plan_destroy.restype = None
        L.pm_batch_polymul.argtypes = [P(pm_batch_item), C.c_uint32, P(pm_batch_options), P(pm_batch_stats),
                                       C.c_void_p]
        L.pm_batch_polymul.restype = C.c_int
        L.pm_batch_workspace.argtypes = [P(pm_batch_item), C.c_uint32, P(pm_batch_options), P(C.c_uint64),
                                         P(C.c_uint64)]
        L.pm_batch_workspace.restype = C.c_int
        _batch_ready = True
    return L


def batch_workspace(products, range_target: int = 0, ranges_per_item: int = 0):
    """(device bytes, host bytes) the batched pass needs for `products`
    (pm_batch_workspace; host arithmetic only)."""
    n = len(products)
    items = (pm_batch_item * n)()
    for k, pr in enumerate(products):
        items[k] = _batch_item(pr)
    opt = pm_batch_options(range_target, ranges_per_item)
    d, h = C.c_uint64(0), C.c_uint64(0)
    rc = _batch_lib().pm_batch_workspace(items, n, C.byref(opt), C.byref(d), C.byref(h))
    if rc != PM_OK:
        raise PolymulError(rc, "pm_batch_workspace")
    return int(d.value), int(h.value)


class BatchPlan:
    """A batch of products captured once into a CUDA graph.

    ``products``: list of dicts with keys field_bits, kind ('m61'/'i64'),
    f_exps, f_coefs, g_exps, g_coefs (CUDA tensors) and out = (keys, coefs)
    CUDA tensors (their length is the capacity).  The tensors must stay alive
    and unmoved while the plan exists."""

    def __init__(self, products, range_target: int = 0, ranges_per_item: int = 0, stream=None):
        self.products = products
        n = len(products)
        self.items = (pm_batch_item * n)()
        for k, pr in enumerate(products):
            self.items[k] = _batch_item(pr)
        self.opt = pm_batch_options(range_target, ranges_per_item)
        self.handle = C.c_void_p()
        rc = _batch_lib().pm_batch_plan_create(self.items, n, C.byref(self.opt), C.byref(self.handle),
                                               _stream_handle(stream))
        if rc != PM_OK:
            raise PolymulError(rc, "pm_batch_plan_create")

    def run(self, stream=None):
        rc = _batch_lib().pm_batch_plan_run(self.handle, _stream_handle(stream))
        if rc != PM_OK:
            raise PolymulError(rc, "pm_batch_plan_run")

    def finish(self, stream=None):
        """Returns (list of (status, n) per product, stats dict)."""
        st = pm_batch_stats()
        _batch_lib().pm_batch_plan_finish(self.handle, self.items, C.byref(st), _stream_handle(stream))
        return [(int(it.status), int(it.h.n)) for it in self.items], st.as_dict()

    def close(self):
        if self.handle:
            _batch_lib().pm_batch_plan_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_polymul(products, range_target: int = 0, ranges_per_item: int = 0, stream=None):
    """One-shot batch: create, run, finish, destroy."""
    plan = BatchPlan(products, range_target, ranges_per_item, stream)
    try:
        plan.run(stream)
        return plan.finish(stream)
    finally:
        plan.close()


# ---------------------------------------------------------------------------
# serving engine (pm_server_*)
# ---------------------------------------------------------------------------

class pm_server_config(C.Structure):
    _fields_ = [("device_budget", C.c_uint64), ("host_budget", C.c_uint64), ("streams", C.c_uint32),
                ("max_batch", C.c_uint32), ("batch", pm_batch_options)]


class pm_server_done(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("status", C.c_int32), ("pad", C.c_uint32), ("n", C.c_uint64),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double)]


class pm_server_state_t(C.Structure):
    _fields_ = [("queued", C.c_uint32), ("in_flight", C.c_uint32), ("big_queued", C.c_uint32),
                ("big_active", C.c_uint32), ("max_in_flight", C.c_uint32), ("pad", C.c_uint32),
                ("batches", C.c_uint64), ("device_used", C.c_uint64), ("clock", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


_server_ready = False


def _server_lib():
    global _server_ready
    L = _batch_lib()
    if not _server_ready:
        P = C.POINTER
        L.pm_server_create.argtypes = [P(pm_server_config), P(C.c_void_p)]
        L.pm_server_create.restype = C.c_int
        L.pm_server_submit.argtypes = [C.c_void_p, P(pm_batch_item), C.c_uint64]
        L.pm_server_submit.restype = C.c_int
        L.pm_server_cancel.argtypes = [C.c_void_p, C.c_uint64]
        L.pm_server_cancel.restype = C.c_int
        L.pm_server_progress.argtypes = [C.c_void_p, P(pm_server_done), C.c_uint32, P(C.c_uint32)]
        L.pm_server_progress.restype = C.c_int
        L.pm_server_state.argtypes = [C.c_void_p, P(pm_server_state_t)]
        L.pm_server_state.restype = C.c_int
        L.pm_server_destroy.argtypes = [C.c_void_p]
        L.pm_server_destroy.restype = None
        _server_ready = True
    return L


def _batch_item(pr) -> pm_batch_item:
    kind = pr.get("kind", "m61")
    check_operands(pr["field_bits"], pr["f_exps"], pr["f_coefs"], pr["g_exps"], pr["g_coefs"], kind)
    check_out(pr["out"], kind)
    _check_cuda(pr["f_exps"], pr["f_coefs"], pr["g_exps"], pr["g_coefs"], pr["out"][0], pr["out"][1])
    it = pm_batch_item()
    it.pk = packing(pr["field_bits"])
    it.coef_kind = KIND[pr.get("kind", "m61")]
    it.f = _terms_in(pr["f_exps"], pr["f_coefs"])
    it.g = _terms_in(pr["g_exps"], pr["g_coefs"])
    it.h.keys = pr["out"][0].data_ptr()
    it.h.coefs = pr["out"][1].data_ptr()
    it.h.cap = int(pr["out"][0].shape[0])
    return it


class Server:
    """The native continuous-batching engine (pm_server_*)."""

    def __init__(self, device_budget: int = 0, host_budget: int = 0, streams: int = 0, max_batch: int = 0,
                 range_target: int = 0, ranges_per_item: int = 0):
        cfg = pm_server_config(device_budget, host_budget, streams, max_batch,
                               pm_batch_options(range_target, ranges_per_item))
        self.handle = C.c_void_p()
        rc = _server_lib().pm_server_create(C.byref(cfg), C.byref(self.handle))
        if rc != PM_OK:
            raise PolymulError(rc, "pm_server_create")
        self._buf = (pm_server_done * 4096)()

    def submit(self, product, tag: int):
        it = _batch_item(product)
        rc = _server_lib().pm_server_submit(self.handle, C.byref(it), tag)
        if rc != PM_OK:
            raise PolymulError(rc, "pm_server_submit")

    def cancel(self, tag: int) -> bool:
        """Withdraw a request not yet admitted (True), else False."""
        return _server_lib().pm_server_cancel(self.handle, tag) == PM_OK

    def progress(self):
        n = C.c_uint32()
        rc = _server_lib().pm_server_progress(self.handle, self._buf, len(self._buf), C.byref(n))
        if rc != PM_OK:
            raise PolymulError(rc, "pm_server_progress")
        return [dict(tag=int(d.tag), status=int(d.status), n=int(d.n), t_submit=d.t_submit, t_admit=d.t_admit,
                     t_done=d.t_done) for d in self._buf[:n.value]]

    def state(self):
        st = pm_server_state_t()
        _server_lib().pm_server_state(self.handle, C.byref(st))
        return st.as_dict()

    def close(self):
        if self.handle:
            _server_lib().pm_server_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# autotuner (pm_autotune, pm_batch_autotune)
# ---------------------------------------------------------------------------

PM_TUNE_MAX_CANDIDATES = 24


class pm_tune_report(C.Structure):
    _fields_ = [("count", C.c_uint32), ("best", C.c_uint32), ("candidates", pm_options * PM_TUNE_MAX_CANDIDATES),
                ("ms", C.c_float * PM_TUNE_MAX_CANDIDATES)]


class pm_batch_tune_report(C.Structure):
    _fields_ = [("count", C.c_uint32), ("best", C.c_uint32), ("sample", C.c_uint32),
                ("candidates", pm_batch_options * PM_TUNE_MAX_CANDIDATES), ("ms", C.c_float * PM_TUNE_MAX_CANDIDATES)]


def _opts_dict(o: pm_options) -> dict:
    return dict(strategy=STRATEGY_NAME.get(o.strategy, o.strategy), slots=o.slots, chunk=o.chunk,
                ranges_per_sm=o.ranges_per_sm, accumulator={v: k for k, v in ACCUMULATOR.items()}.get(o.accumulator),
                cost_row=o.cost_row, cost_window=o.cost_window, grid_l=o.grid_l)


def autotune(field_bits, f_exps, f_coefs, g_exps, g_coefs, kind: str = "m61", stream=None):
    """Time every candidate configuration on this product, keep the fastest
    for its shape class (later pm_polymul calls with default options use it)
    and return (best options dict, [(options dict, ms)])."""
    import torch
    _check_cuda(f_exps, f_coefs, g_exps, g_coefs)
    L = lib()
    L.pm_autotune.argtypes = [C.POINTER(pm_packing), C.c_int, C.POINTER(pm_terms_in), C.POINTER(pm_terms_in),
                              C.POINTER(pm_terms_out), C.POINTER(pm_options), C.POINTER(pm_tune_report), C.c_void_p]
    L.pm_autotune.restype = C.c_int
    cap = out_bound(field_bits, f_exps, g_exps, stream)
    words = {"m61": 1, "i64": 2, "i192": 3}[kind]
    keys = torch.empty(max(cap, 1), dtype=torch.int64, device=f_exps.device)
    coefs = torch.empty((max(cap, 1), words) if words > 1 else (max(cap, 1),), dtype=torch.int64,
                        device=f_exps.device)
    h = pm_terms_out(keys.data_ptr(), coefs.data_ptr(), 0, cap)
    best = pm_options()
    rep = pm_tune_report()
    pk = packing(field_bits)
    f = _terms_in(f_exps, f_coefs)
    g = _terms_in(g_exps, g_coefs)
    rc = L.pm_autotune(C.byref(pk), KIND[kind], C.byref(f), C.byref(g), C.byref(h), C.byref(best), C.byref(rep),
                       _stream_handle(stream))
    if rc != PM_OK:
        raise PolymulError(rc, "pm_autotune")
    table = [(_opts_dict(rep.candidates[k]), float(rep.ms[k])) for k in range(rep.count)]
    return _opts_dict(best), table


def batch_autotune(products, stream=None):
    """Pick (range_target, ranges_per_item) for a batch by timing plans on a
    sample of it; returns (best dict, [(candidate dict, ms)])."""
    L = _batch_lib()
    L.pm_batch_autotune.argtypes = [C.POINTER(pm_batch_item), C.c_uint32, C.POINTER(pm_batch_options),
                                    C.POINTER(pm_batch_tune_report), C.c_void_p]
    L.pm_batch_autotune.restype = C.c_int
    n = len(products)
    items = (pm_batch_item * n)()
    for k, pr in enumerate(products):
        items[k] = _batch_item(pr)
    best = pm_batch_options()
    rep = pm_batch_tune_report()
    rc = L.pm_batch_autotune(items, n, C.byref(best), C.byref(rep), _stream_handle(stream))
    if rc != PM_OK:
        raise PolymulError(rc, "pm_batch_autotune")
    table = [({"range_target": rep.candidates[k].range_target, "ranges_per_item": rep.candidates[k].ranges_per_item},
              float(rep.ms[k])) for k in range(rep.count)]
    return {"range_target": best.range_target, "ranges_per_item": best.ranges_per_item}, table

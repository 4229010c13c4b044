"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

This module only draws random numbers and enumerates exponent sets.  It holds
none of the product's arithmetic (no packing, no coefficient products, no
combining of terms): both implementations receive the same arrays from here
and compute everything else on their own.

Random numbers come from the SplitMix64 sequence (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): the k-th
output of a stream with state s is mix(s + k * 0x9E3779B97F4A7C15).  Because
the sequence is counter based it vectorises in numpy and gives the same
numbers on every machine.

Workload shapes follow the sparse distributed format of Sec. 2 (a list of
(coefficient, exponent vector) terms) and the five workloads the library is
measured on:

  workload_sparse4v      4 variables, 1000 + 1000 distinct terms of total
                         degree <= 12
  workload_dense4v       4 variables, all 10,626 monomials of total degree
                         <= 20 on both sides
  workload_sparse5v      5 variables, 50,000 + 50,000 distinct terms, degree
                         caps (6,8,10,12,16)
  workload_sparse_batch  4096 independent products, 3..8 variables,
                         log-uniform sizes [16,4096]
  workload_serving_mix   a Poisson request stream mixing batch-shaped and
                         dense 4-variable products
"""

from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

P61 = (1 << 61) - 1           # the Mersenne prime 2^61 - 1
GOLDEN = np.uint64(0x9E3779B97F4A7C15)
BASE_SEED = 0x130374250000    # workload seeds are BASE_SEED + workload index

_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


class Stream:
    """One SplitMix64 stream.  ``Stream(seed, sid)`` derives independent
    streams (one per operand, per request, ...) from one workload seed."""

    def __init__(self, seed: int, sid: int = 0):
        s0 = np.array([(seed + sid * 0x6A09E667F3BCC909) & (2**64 - 1)], dtype=np.uint64)
        self.state = int(_mix(s0)[0])

    def u64(self, n: int) -> np.ndarray:
        if n <= 0:
            return np.zeros(0, dtype=np.uint64)
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = np.uint64(self.state) + k * GOLDEN
        self.state = (self.state + n * int(GOLDEN)) & (2**64 - 1)
        return _mix(z)

    def below(self, m: int, n: int) -> np.ndarray:
        """n integers in [0, m) (modulo reduction; bias <= m / 2^64)."""
        if m <= 0:
            raise ValueError("m must be positive")
        return (self.u64(n) % np.uint64(m)).astype(np.uint64)

    def uniform01(self, n: int) -> np.ndarray:
        return (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / float(1 << 53))

    def coef_m61(self, n: int) -> np.ndarray:
        """n coefficients uniform in [1, p), p = 2^61 - 1 (zeros redrawn)."""
        out = self.u64(n) >> np.uint64(3)
        bad = (out == 0) | (out >= np.uint64(P61))
        while bad.any():
            out[bad] = self.u64(int(bad.sum())) >> np.uint64(3)
            bad = (out == 0) | (out >= np.uint64(P61))
        return out

    def coef_i64(self, n: int, bound: int) -> np.ndarray:
        """n int64 coefficients uniform in [-bound, bound] minus {0}."""
        out = self.below(2 * bound + 1, n).astype(np.int64) - bound
        bad = out == 0
        while bad.any():
            out[bad] = self.below(2 * bound + 1, int(bad.sum())).astype(np.int64) - bound
            bad = out == 0
        return out

    def permutation(self, n: int) -> np.ndarray:
        return np.argsort(self.u64(n), kind="stable")


# --------------------------------------------------------------------------
# exponent sets
# --------------------------------------------------------------------------

def monomials_total_degree(nvars: int, d: int) -> np.ndarray:
    """All exponent vectors with sum <= d, shape (C(nvars+d, nvars), nvars)."""
    rows = [e for e in itertools.product(range(d + 1), repeat=nvars) if sum(e) <= d]
    return np.array(rows, dtype=np.uint32).reshape(-1, nvars)


def box_points(caps: Sequence[int]) -> np.ndarray:
    """All exponent vectors with 0 <= e_v <= caps[v]."""
    grids = np.meshgrid(*[np.arange(c + 1, dtype=np.uint32) for c in caps], indexing="ij")
    return np.stack([g.reshape(-1) for g in grids], axis=1).astype(np.uint32)


def distinct_random_vectors(st: Stream, n: int, nvars: int, hi: int) -> np.ndarray:
    """n distinct exponent vectors, each entry uniform in [0, hi]."""
    out = np.zeros((0, nvars), dtype=np.uint32)
    while out.shape[0] < n:
        need = n - out.shape[0]
        cand = st.below(hi + 1, need * nvars).astype(np.uint32).reshape(need, nvars)
        both = np.concatenate([out, cand], axis=0)
        _, first = np.unique(both, axis=0, return_index=True)
        out = both[np.sort(first)]
    return out[:n]


# --------------------------------------------------------------------------
# polynomials as plain arrays
# --------------------------------------------------------------------------

@dataclass
class Poly:
    exps: np.ndarray          # (n, nvars) uint32, row-major
    coefs: np.ndarray         # (n,) uint64 (mod-p kind) or int64 (int64 kind)

    @property
    def n(self) -> int:
        return int(self.exps.shape[0])

    @property
    def nvars(self) -> int:
        return int(self.exps.shape[1])


@dataclass
class Workload:
    name: str
    nvars: int
    field_bits: List[int]
    kind: str                 # "m61" or "i64"
    f: Poly
    g: Poly
    note: str = ""

    @property
    def term_products(self) -> int:
        return self.f.n * self.g.n


def default_field_bits(nvars: int) -> List[int]:
    w = 64 // nvars
    return [w] * nvars


def _poly(st: Stream, exps: np.ndarray, kind: str, i64_bound: int = 1 << 20) -> Poly:
    order = st.permutation(exps.shape[0])       # terms arrive unsorted
    exps = np.ascontiguousarray(exps[order])
    if kind == "m61":
        c = st.coef_m61(exps.shape[0])
    else:
        c = st.coef_i64(exps.shape[0], i64_bound)
    return Poly(exps, c)


def workload_sparse4v(seed: Optional[int] = None) -> Workload:
    seed = BASE_SEED + 0 if seed is None else seed
    mons = monomials_total_degree(4, 12)                 # 1820 monomials
    out = []
    for sid in (0, 1):
        st = Stream(seed, sid)
        pick = st.permutation(mons.shape[0])[:1000]
        out.append(_poly(st, mons[pick], "m61"))
    return Workload("sparse4v_1000x1000_m61", 4, [16] * 4, "m61", out[0], out[1],
                    "4 vars, 16-bit fields, 1000 distinct terms of degree <= 12 per operand")


def workload_dense4v(kind: str = "m61", seed: Optional[int] = None) -> Workload:
    seed = BASE_SEED + 1 if seed is None else seed
    mons = monomials_total_degree(4, 20)                 # 10626 monomials
    out = []
    for sid in (0, 1):
        st = Stream(seed, sid + (2 if kind == "i64" else 0))
        out.append(_poly(st, mons, kind))
    return Workload(f"dense4v_deg20_{kind}", 4, [16] * 4, kind, out[0], out[1],
                    "4 vars, all 10626 monomials of degree <= 20 on both sides")


def paper_example1() -> Workload:
    """Sec. 6, Example 1: f1 = (1 + x + y + z + t)^40 and g1 = f1 + 1, 135,751
    terms each, coefficients mod 2^61 - 1 (the multinomial expansion; no
    random draws)."""
    e, c = multinomial_power(4, 40)
    fc = np.array(c, dtype=np.uint64)
    gc = fc.copy()
    const = int(np.flatnonzero((e == 0).all(axis=1))[0])
    gc[const] = (int(gc[const]) + 1) % P61
    return Workload("paper_ex1_4v_pow40", 4, [16] * 4, "m61", Poly(e, fc), Poly(e.copy(), gc),
                    "f1 = (1+x+y+z+t)^40, g1 = f1 + 1 (135,751 terms each)")


def paper_example(name: str, power: Optional[int] = None) -> Workload:
    """Sec. 6, Examples 1-3, coefficients mod 2^61 - 1 (multinomial
    expansions; no random draws):
      ex1: (1+x+y+z+t)^40 times itself plus one (4 variables);
      ex2: (1+x+y+2z^2+3t^3+5u^5)^25 times (1+u+t+2z^2+3y^3+5x^5)^25;
      ex3: (1+u^2+v+w^2+x-y^2)^28 times (1+u+v^2+w+x^2+y^3)^28 + 1.
    Variables in the order written (x_1 first).  `power` (Examples 2 and 3
    only) replaces the paper's exponent 25 or 28 by a smaller one: the same
    shape at a size that profiles quickly."""
    if name == "ex1":
        return paper_example1()
    if name == "ex2":
        k = 25 if power is None else power
        fe, fcl = multinomial_power(5, k, [(1, 1), (1, 1), (2, 2), (3, 3), (5, 5)])
        ge, gcl = multinomial_power(5, k, [(5, 5), (3, 3), (2, 2), (1, 1), (1, 1)])
        bits = [12] * 5                     # exponents up to 150 per variable
        desc = f"(1+x+y+2z^2+3t^3+5u^5)^{k} x (1+u+t+2z^2+3y^3+5x^5)^{k}"
    elif name == "ex3":
        k = 28 if power is None else power
        fe, fcl = multinomial_power(5, k, [(1, 2), (1, 1), (1, 2), (1, 1), (-1, 2)])
        ge, gcl = multinomial_power(5, k, [(1, 1), (1, 2), (1, 1), (1, 2), (1, 3)])
        const = int(np.flatnonzero((ge == 0).all(axis=1))[0])
        gcl[const] = (gcl[const] + 1) % P61
        bits = [12] * 5                     # exponents up to 140 per variable
        desc = f"(1+u^2+v+w^2+x-y^2)^{k} x ((1+u+v^2+w+x^2+y^3)^{k} + 1)"
    else:
        raise ValueError(name)
    if k > (25 if name == "ex2" else 28) or k < 1:
        raise ValueError("power above the paper's or below 1")
    f = Poly(fe, np.array(fcl, dtype=np.uint64))
    g = Poly(ge, np.array(gcl, dtype=np.uint64))
    return Workload(f"paper_{name}", 5, bits, "m61", f, g, desc)


C3_CAPS = (6, 8, 10, 12, 16)


def workload_sparse5v(seed: Optional[int] = None, n: int = 50000) -> Workload:
    seed = BASE_SEED + 2 if seed is None else seed
    pts = box_points(C3_CAPS)                            # 153153 points
    out = []
    for sid in (0, 1):
        st = Stream(seed, sid)
        pick = st.permutation(pts.shape[0])[:n]
        out.append(_poly(st, pts[pick], "m61"))
    return Workload(f"sparse5v_{n}x{n}_m61", 5, [12] * 5, "m61", out[0], out[1],
                    "5 vars, degree caps (6,8,10,12,16), 12-bit fields")


def log_uniform_size(st: Stream, count: int, lo: int = 16, hi: int = 4096) -> np.ndarray:
    u = st.uniform01(count)
    n = np.floor(lo * np.exp(u * math.log(hi / lo))).astype(np.int64)
    return np.clip(n, lo, hi)


def sparse_product(st: Stream, nvars: int, nf: int, ng: int, exp_hi: Optional[int] = None) -> Workload:
    bits = default_field_bits(nvars)
    if exp_hi is None:
        exp_hi = (1 << (bits[0] - 2)) - 1
    fe = distinct_random_vectors(st, nf, nvars, exp_hi)
    ge = distinct_random_vectors(st, ng, nvars, exp_hi)
    f = Poly(fe, st.coef_m61(nf))
    g = Poly(ge, st.coef_m61(ng))
    return Workload(f"sparse{nvars}v_{nf}x{ng}", nvars, bits, "m61", f, g)


def workload_sparse_batch(count: int = 4096, seed: Optional[int] = None,
                exp_hi: Optional[int] = None) -> List[Workload]:
    """The batched workload: ``count`` independent sparse products."""
    seed = BASE_SEED + 3 if seed is None else seed
    st = Stream(seed, 0)
    nv = 3 + st.below(6, count).astype(np.int64)
    nf = log_uniform_size(st, count)
    ng = log_uniform_size(st, count)
    out = []
    for k in range(count):
        sk = Stream(seed, 1 + k)
        out.append(sparse_product(sk, int(nv[k]), int(nf[k]), int(ng[k]), exp_hi))
    return out


@dataclass
class Request:
    t_arrival: float          # seconds from stream start
    work: Workload
    dense: bool


def workload_serving_mix(rate_hz: float, count: int, seed: Optional[int] = None,
                dense_frac: float = 0.05) -> List[Request]:
    """Poisson arrivals; 95% products drawn like workload_sparse_batch's, 5%
    dense 4-variable ones of workload_dense4v's shape."""
    seed = BASE_SEED + 4 if seed is None else seed
    st = Stream(seed, 0)
    gaps = -np.log(1.0 - st.uniform01(count)) / rate_hz
    t = np.cumsum(gaps)
    kinds = st.uniform01(count) < dense_frac
    nv = 3 + st.below(6, count).astype(np.int64)
    nf = log_uniform_size(st, count)
    ng = log_uniform_size(st, count)
    mons = None
    reqs = []
    for k in range(count):
        sk = Stream(seed, 1 + k)
        if kinds[k]:
            if mons is None:
                mons = monomials_total_degree(4, 20)
            f = _poly(sk, mons, "m61")
            g = _poly(sk, mons, "m61")
            w = Workload("dense4v_deg20", 4, [16] * 4, "m61", f, g)
        else:
            w = sparse_product(sk, int(nv[k]), int(nf[k]), int(ng[k]))
        reqs.append(Request(float(t[k]), w, bool(kinds[k])))
    return reqs


# --------------------------------------------------------------------------
# closed-form operands (pins): multinomial expansions, no products computed
# --------------------------------------------------------------------------

def multinomial_power(nvars: int, k: int, weights: Optional[Sequence[Tuple[int, int]]] = None,
                      mod: Optional[int] = P61) -> Tuple[np.ndarray, List[int]]:
    """Expansion of (c_0 + c_1 x_{v_1}^{d_1} + ...)^k by the multinomial theorem.

    ``weights`` lists (coefficient, degree) for each variable x_1..x_nvars
    (default: all (1, 1), i.e. (1 + x_1 + ... + x_n)^k).  The constant term
    is 1.  Returns (exps, coefs) with Python-int coefficients (reduced mod
    ``mod`` when given).
    """
    if weights is None:
        weights = [(1, 1)] * nvars
    exps, coefs = [], []
    for ks in itertools.product(range(k + 1), repeat=nvars):
        s = sum(ks)
        if s > k:
            continue
        c = math.factorial(k) // math.factorial(k - s)
        for kv in ks:
            c //= math.factorial(kv)
        for (w, _), kv in zip(weights, ks):
            c *= w ** kv
        exps.append([d * kv for (_, d), kv in zip(weights, ks)])
        coefs.append(c % mod if mod else c)
    return np.array(exps, dtype=np.uint32).reshape(-1, nvars), coefs

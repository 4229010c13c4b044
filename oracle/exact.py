"""The product by its definition in Python integers, for int64 coefficients
of any size: the reference for the 192-bit accumulation kind.

TEST INFRASTRUCTURE ONLY: the tests use this module; the library never
does.  Plain loops over all term pairs, so small and medium cases only.

h = sum_{i,j} a_i b_j x^(alpha_i + beta_j) (Sec. 2), with the input
conventions of the library: repeated input monomials are summed (a sum that
leaves int64 is refused, like the library's rule for int64 inputs), zero
coefficients are dropped, every exponent must stay below its field's guard
bit 2^(w_v - 1) in the inputs and in the product, and the result is sorted
by the monomial order with x_1 most significant -- lexicographic order of
the exponent tuples.  Coefficients are exact Python integers, returned as
three 64-bit two's complement words (low word first).
"""

from __future__ import annotations

from typing import Dict, Sequence, Tuple

import numpy as np

OR_EEXP_OVERFLOW, OR_ECOEF_BOUND = -2, -3


class ExactError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"exact product error {code}")
        self.code = code


def _canonical(exps, coefs, nvars: int, limits) -> Dict[Tuple[int, ...], int]:
    terms: Dict[Tuple[int, ...], int] = {}
    for e, c in zip(np.asarray(exps, dtype=np.int64).reshape(-1, nvars).tolist(),
                    np.asarray(coefs, dtype=np.int64).tolist()):
        if any(x >= lim for x, lim in zip(e, limits)):
            raise ExactError(OR_EEXP_OVERFLOW)
        k = tuple(e)
        terms[k] = terms.get(k, 0) + int(c)
    for v in terms.values():
        if v > 2**63 - 1 or v < -2**63:
            raise ExactError(OR_ECOEF_BOUND)
    return {k: v for k, v in terms.items() if v != 0}


def words192(v: int) -> Tuple[int, int, int]:
    """v as three 64-bit two's complement words, low word first."""
    u = v % (1 << 192)
    return u & (2**64 - 1), (u >> 64) & (2**64 - 1), u >> 128


def mul_exact(nvars: int, field_bits: Sequence[int], fe, fc, ge, gc) -> Tuple[np.ndarray, np.ndarray]:
    """Returns (exps (n, nvars) uint32, coefs (n, 3) uint64 words)."""
    limits = [1 << (w - 1) for w in field_bits]
    F = _canonical(fe, fc, nvars, limits)
    G = _canonical(ge, gc, nvars, limits)
    if F and G:
        for v in range(nvars):
            if max(k[v] for k in F) + max(k[v] for k in G) >= limits[v]:
                raise ExactError(OR_EEXP_OVERFLOW)
    h: Dict[Tuple[int, ...], int] = {}
    for ka, a in F.items():
        for kb, b in G.items():
            k = tuple(x + y for x, y in zip(ka, kb))
            h[k] = h.get(k, 0) + a * b
    keys = sorted(k for k, v in h.items() if v != 0)
    e = np.array(keys, dtype=np.uint32).reshape(-1, nvars)
    c = np.array([words192(h[k]) for k in keys], dtype=np.uint64).reshape(-1, 3)
    return e, c

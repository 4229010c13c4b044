"""Pins for the oracle: checks against what the paper and the mathematics fix,
never against the oracle itself.

 - brute force: dense mixed-radix array convolution on tiny inputs (a
   different algorithm from the oracle's hash map);
 - closed forms: (1+x_1+..+x_n)^a (1+..+x_n)^b = (1+..+x_n)^(a+b) with
   multinomial coefficients; dense degree-d times degree-e operands give
   C(n+d+e, n) terms; the paper's printed term counts (Sec. 6);
 - evaluation at random points mod p (Schwartz-Zippel), done in Python ints;
 - invariants: commutativity, identity, monomial shift, distributivity;
 - int128 results near the 2^127 bound, and the error rules;
 - the Sec. 5 grid against a hand-derived fixture; Alg. 1 against the
   definition.
"""

import math
import os
import random

import numpy as np
import pytest

import oracle
import polygen
from polygen import P61

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# test-side helpers (independent of oracle.c)
# ---------------------------------------------------------------------------

def dense_convolution(nv, fe, fc, ge, gc, mod=P61):
    """Product by dense arrays: place every term of f at its exponent in an
    array, then add shifted copies of g's array.  Returns {exp tuple: coef}."""
    fe = np.asarray(fe, dtype=np.int64).reshape(-1, nv)
    ge = np.asarray(ge, dtype=np.int64).reshape(-1, nv)
    df = tuple(int(fe[:, v].max()) + 1 if len(fe) else 1 for v in range(nv))
    dg = tuple(int(ge[:, v].max()) + 1 if len(ge) else 1 for v in range(nv))
    F = np.zeros(df, dtype=object); F[...] = 0
    G = np.zeros(dg, dtype=object); G[...] = 0
    for e, c in zip(fe, fc):
        F[tuple(e)] += int(c)
    for e, c in zip(ge, gc):
        G[tuple(e)] += int(c)
    H = np.zeros(tuple(a + b - 1 for a, b in zip(df, dg)), dtype=object); H[...] = 0
    for idx in np.ndindex(*df):
        a = F[idx]
        if a == 0:
            continue
        sl = tuple(slice(i, i + d) for i, d in zip(idx, dg))
        H[sl] = H[sl] + a * G
    out = {}
    for idx in np.ndindex(*H.shape):
        v = H[idx] % mod if mod else H[idx]
        if v != 0:
            out[tuple(int(i) for i in idx)] = int(v)
    return out


def as_dict(exps, coefs, kind="m61"):
    if kind == "m61":
        return {tuple(int(x) for x in e): int(c) for e, c in zip(exps, coefs)}
    vals = oracle.i128_to_int(coefs)
    return {tuple(int(x) for x in e): v for e, v in zip(exps, vals)}


def is_lex_sorted_strict(exps):
    rows = [tuple(int(x) for x in e) for e in exps]
    return all(rows[i] < rows[i + 1] for i in range(len(rows) - 1))


def eval_py(exps, coefs, r, mod=P61):
    acc = 0
    for e, c in zip(exps, coefs):
        t = int(c) % mod
        for v, x in enumerate(e):
            t = t * pow(int(r[v]), int(x), mod) % mod
        acc = (acc + t) % mod
    return acc


def random_poly(rng, nv, n, maxdeg, kind="m61", dup=True, zeros=True):
    exps = rng.integers(0, maxdeg + 1, size=(n, nv)).astype(np.uint32)
    if kind == "m61":
        coefs = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, size=n, dtype=np.uint64)
    else:
        coefs = rng.integers(-2**40, 2**40, size=n, dtype=np.int64)
    if zeros and n > 2:
        coefs[1] = 0
    if dup and n > 3:
        exps[3] = exps[0]
    return exps, coefs


BITS4 = [16, 16, 16, 16]


# ---------------------------------------------------------------------------
# brute force
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("nv,maxdeg,nf,ng,seed", [
    (1, 6, 5, 7, 1), (2, 6, 12, 9, 2), (3, 4, 20, 25, 3), (3, 6, 40, 30, 4), (2, 3, 1, 16, 5),
])
def test_bruteforce_m61(nv, maxdeg, nf, ng, seed):
    rng = np.random.default_rng(seed)
    fe, fc = random_poly(rng, nv, nf, maxdeg)
    ge, gc = random_poly(rng, nv, ng, maxdeg)
    he, hc = oracle.mul(nv, [8] * nv, "m61", fe, fc, ge, gc)
    assert is_lex_sorted_strict(he)
    assert np.all(hc != 0) and np.all(hc < P61)
    assert as_dict(he, hc) == dense_convolution(nv, fe, fc, ge, gc)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_bruteforce_i64(seed):
    rng = np.random.default_rng(seed)
    fe, fc = random_poly(rng, 3, 30, 5, kind="i64")
    ge, gc = random_poly(rng, 3, 25, 5, kind="i64")
    he, hc = oracle.mul(3, [8] * 3, "i64", fe, fc, ge, gc)
    assert is_lex_sorted_strict(he)
    assert as_dict(he, hc, "i64") == dense_convolution(3, fe, fc, ge, gc, mod=None)


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n,a,b", [(3, 4, 5), (4, 3, 3), (2, 7, 0), (1, 9, 4), (5, 2, 3)])
def test_power_of_linear_form(n, a, b):
    fe, fc = polygen.multinomial_power(n, a)
    ge, gc = polygen.multinomial_power(n, b)
    he, hc = oracle.mul(n, [12] * n, "m61", fe, np.array(fc, dtype=np.uint64), ge,
                        np.array(gc, dtype=np.uint64))
    assert len(he) == math.comb(n + a + b, n)
    ee, ec = polygen.multinomial_power(n, a + b)
    assert as_dict(he, hc) == {tuple(int(x) for x in e): int(c) for e, c in zip(ee, ec)}


@pytest.mark.parametrize("n,d,e", [(2, 5, 7), (3, 4, 6), (4, 3, 5)])
def test_dense_total_degree_count(n, d, e):
    st = polygen.Stream(99, n)
    F = polygen.monomials_total_degree(n, d)
    G = polygen.monomials_total_degree(n, e)
    fc = (st.below(1000, len(F)) + 1).astype(np.int64)   # positive: no cancellation
    gc = (st.below(1000, len(G)) + 1).astype(np.int64)
    he, hc = oracle.mul(n, [12] * n, "i64", F, fc, G, gc)
    assert len(he) == math.comb(n + d + e, n)
    assert all(v > 0 for v in oracle.i128_to_int(hc))


def _read_counts():
    rows = {}
    with open(os.path.join(GOLDEN, "paper_counts.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                name, k, nop, nres = line.split()
                rows[name] = (int(k), int(nop), int(nres))
    return rows


def test_paper_example1_counts():
    """Ex. 1: f1 = (1+x+y+z+t)^k, g1 = f1 + 1.  The closed-form counts
    C(k+4,4) and C(2k+4,4) reproduce the paper's printed numbers at k = 40,
    and the oracle reproduces the closed form at small k."""
    k, nop, nres = _read_counts()["ex1"]
    assert math.comb(k + 4, 4) == nop and math.comb(2 * k + 4, 4) == nres
    for kk in (2, 3, 4):
        fe, fc = polygen.multinomial_power(4, kk)
        gc = list(fc)
        gc[0] = (gc[0] + 1) % P61          # the constant term of f1 + 1
        he, hc = oracle.mul(4, BITS4, "m61", fe, np.array(fc, dtype=np.uint64), fe,
                            np.array(gc, dtype=np.uint64))
        assert len(he) == math.comb(2 * kk + 4, 4)


EX2_F = [(1, 1), (1, 1), (2, 2), (3, 3), (5, 5)]      # 1 + x + y + 2z^2 + 3t^3 + 5u^5
EX2_G = [(5, 5), (3, 3), (2, 2), (1, 1), (1, 1)]      # 1 + u + t + 2z^2 + 3y^3 + 5x^5
EX3_F = [(1, 2), (1, 1), (1, 2), (1, 1), (-1, 2)]     # 1 + u^2 + v + w^2 + x - y^2
EX3_G = [(1, 1), (1, 2), (1, 1), (1, 2), (1, 3)]      # 1 + u + v^2 + w + x^2 + y^3


def test_paper_example2_3_operand_counts():
    """Operand counts of Ex. 2 and Ex. 3: C(k+5,5) at the printed powers."""
    c = _read_counts()
    assert math.comb(c["ex2"][0] + 5, 5) == c["ex2"][1]
    assert math.comb(c["ex3"][0] + 5, 5) == c["ex3"][1]
    for w in (EX2_F, EX2_G, EX3_F, EX3_G):
        e, _ = polygen.multinomial_power(5, 4, w)
        assert len(e) == math.comb(4 + 5, 5) and len({tuple(r) for r in e}) == len(e)


@pytest.mark.parametrize("k", [2, 3])
def test_paper_example2_small_power(k):
    fe, fc = polygen.multinomial_power(5, k, EX2_F)
    ge, gc = polygen.multinomial_power(5, k, EX2_G)
    fc = np.array(fc, dtype=np.uint64); gc = np.array(gc, dtype=np.uint64)
    he, hc = oracle.mul(5, [12] * 5, "m61", fe, fc, ge, gc)
    assert as_dict(he, hc) == dense_convolution(5, fe, fc, ge, gc)


# ---------------------------------------------------------------------------
# evaluation at random points (Schwartz-Zippel, error <= deg / p)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("kind,seed", [("m61", 1), ("m61", 2), ("i64", 3)])
def test_evaluation_at_points(kind, seed):
    rng = np.random.default_rng(seed)
    fe, fc = random_poly(rng, 4, 300, 9, kind=kind)
    ge, gc = random_poly(rng, 4, 200, 9, kind=kind)
    he, hc = oracle.mul(4, BITS4, kind, fe, fc, ge, gc)
    hv = hc if kind == "m61" else oracle.i128_to_int(hc)
    pr = random.Random(seed)
    for _ in range(3):
        r = [pr.randrange(P61) for _ in range(4)]
        lhs = eval_py(he, hv, r)
        assert lhs == eval_py(fe, fc, r) * eval_py(ge, gc, r) % P61
        # oracle_eval itself is pinned to the Python evaluation
        assert oracle.evaluate(4, "m61" if kind == "m61" else "i128", he, hc, r) == lhs


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

def test_commutative_and_identity_and_shift():
    rng = np.random.default_rng(7)
    fe, fc = random_poly(rng, 3, 120, 7)
    ge, gc = random_poly(rng, 3, 90, 7)
    a = oracle.mul(3, [10] * 3, "m61", fe, fc, ge, gc)
    b = oracle.mul(3, [10] * 3, "m61", ge, gc, fe, fc)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    one_e = np.zeros((1, 3), dtype=np.uint32)
    one_c = np.array([1], dtype=np.uint64)
    ie, ic = oracle.mul(3, [10] * 3, "m61", fe, fc, one_e, one_c)
    canon = {}
    for e, c in zip(fe, fc):
        k = tuple(int(x) for x in e)
        canon[k] = (canon.get(k, 0) + int(c)) % P61
    assert as_dict(ie, ic) == {k: v for k, v in canon.items() if v}
    assert is_lex_sorted_strict(ie)
    m = np.array([[2, 0, 5]], dtype=np.uint32)
    se, sc = oracle.mul(3, [10] * 3, "m61", fe, fc, m, one_c)
    assert np.array_equal(se, ie + m) and np.array_equal(sc, ic)


def test_distributive():
    rng = np.random.default_rng(8)
    fe, fc = random_poly(rng, 2, 60, 8)
    g1e, g1c = random_poly(rng, 2, 40, 8)
    g2e, g2c = random_poly(rng, 2, 50, 8)
    lhs = as_dict(*oracle.mul(2, [10, 10], "m61", fe, fc, np.concatenate([g1e, g2e]),
                              np.concatenate([g1c, g2c])))
    r1 = as_dict(*oracle.mul(2, [10, 10], "m61", fe, fc, g1e, g1c))
    r2 = as_dict(*oracle.mul(2, [10, 10], "m61", fe, fc, g2e, g2c))
    rhs = dict(r1)
    for k, v in r2.items():
        rhs[k] = (rhs.get(k, 0) + v) % P61
    assert lhs == {k: v for k, v in rhs.items() if v}


def test_empty_and_all_zero():
    e = np.zeros((0, 2), dtype=np.uint32)
    c = np.zeros(0, dtype=np.uint64)
    fe = np.array([[1, 2], [3, 4]], dtype=np.uint32)
    he, hc = oracle.mul(2, [8, 8], "m61", fe, np.array([5, 6], dtype=np.uint64), e, c)
    assert he.shape == (0, 2) and hc.shape == (0,)
    he, hc = oracle.mul(2, [8, 8], "m61", fe, np.array([0, P61], dtype=np.uint64), fe,
                        np.array([1, 2], dtype=np.uint64))
    assert he.shape == (0, 2)


# ---------------------------------------------------------------------------
# int128 and the error rules
# ---------------------------------------------------------------------------

def test_int128_large_values_and_cancellation():
    # (2^62 + x)(2^62 - x) = 2^124 - x^2 : the x term cancels
    fe = np.array([[0], [1]], dtype=np.uint32)
    he, hc = oracle.mul(1, [8], "i64", fe, np.array([2**62, 1], dtype=np.int64), fe,
                        np.array([2**62, -1], dtype=np.int64))
    assert as_dict(he, hc, "i64") == {(0,): 2**124, (2,): -1}
    # -2^63 (1 + x) * (2^63 - 1)(1 + x): max|a| max|b| min(n) = 2^127 - 2^64 < 2^127
    a, b = -2**63, 2**63 - 1
    he, hc = oracle.mul(1, [8], "i64", fe, np.array([a, a], dtype=np.int64), fe,
                        np.array([b, b], dtype=np.int64))
    assert as_dict(he, hc, "i64") == {(0,): a * b, (1,): 2 * a * b, (2,): a * b}


def test_int128_bound_rule():
    fe = np.array([[0], [1]], dtype=np.uint32)
    a = -2**63
    with pytest.raises(oracle.OracleError) as ei:          # 2^63 * 2^63 * 2 = 2^127
        oracle.mul(1, [8], "i64", fe, np.array([a, a], dtype=np.int64), fe,
                   np.array([a, 1], dtype=np.int64))
    assert ei.value.code == oracle.OR_ECOEF_BOUND
    # a repeated input monomial whose sum leaves int64
    with pytest.raises(oracle.OracleError) as ei:
        oracle.mul(1, [8], "i64", np.array([[0], [0]], dtype=np.uint32),
                   np.array([2**62, 2**62], dtype=np.int64), fe, np.array([1, 1], dtype=np.int64))
    assert ei.value.code == oracle.OR_ECOEF_BOUND


def test_exponent_guard_rule():
    bits = [4, 4]                                  # exponents must stay < 8
    one = np.array([1], dtype=np.uint64)
    ok = oracle.mul(2, bits, "m61", np.array([[4, 0]], np.uint32), one, np.array([[3, 7]], np.uint32), one)
    assert ok[0].tolist() == [[7, 7]]
    for fe, ge in [([[4, 0]], [[4, 0]]), ([[8, 0]], [[0, 0]]), ([[0, 0]], [[0, 9]])]:
        with pytest.raises(oracle.OracleError) as ei:
            oracle.mul(2, bits, "m61", np.array(fe, np.uint32), one, np.array(ge, np.uint32), one)
        assert ei.value.code == oracle.OR_EEXP_OVERFLOW
    # an input exponent past the guard fails even when its coefficient is zero
    with pytest.raises(oracle.OracleError):
        oracle.mul(2, bits, "m61", np.array([[8, 0], [1, 1]], np.uint32), np.array([0, 1], np.uint64),
                   np.array([[1, 1]], np.uint32), one)


@pytest.mark.parametrize("nv,bits", [(0, []), (17, [2] * 17), (2, [40, 20]), (2, [0, 8]), (3, [30, 30, 8])])
def test_invalid_packing(nv, bits):
    one = np.array([1], dtype=np.uint64)
    e = np.zeros((1, max(nv, 1)), dtype=np.uint32)
    with pytest.raises(oracle.OracleError) as ei:
        oracle.mul(nv, bits or [8], "m61", e, one, e, one)
    assert ei.value.code == oracle.OR_EINVAL


# ---------------------------------------------------------------------------
# Sec. 5 grid and Alg. 1
# ---------------------------------------------------------------------------

def test_grid_matches_hand_derived_fixture():
    want = []
    with open(os.path.join(GOLDEN, "grid_sec5_16x16_l4.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                i, j = line.split()
                want.append((int(i), int(j)))
    alpha = np.arange(1, 17, dtype=np.uint64) * np.uint64(1000)
    beta = np.arange(1, 17, dtype=np.uint64)
    got = [(int(k) // 1000, int(k) % 1000) for k in oracle.grid(alpha, beta, 4)]
    assert sorted(got) == sorted(want)


@pytest.mark.parametrize("l,threads", [(1, 1), (2, 3), (8, 4), (64, 2)])
def test_alg1_equals_definition(l, threads):
    w = polygen.workload_sparse4v()
    ref = oracle.mul(w.nvars, w.field_bits, "m61", w.f.exps[:300], w.f.coefs[:300],
                     w.g.exps[:250], w.g.coefs[:250])
    e, c, ni = oracle.mul_alg1(w.nvars, w.field_bits, "m61", w.f.exps[:300], w.f.coefs[:300],
                               w.g.exps[:250], w.g.coefs[:250], l=l, threads=threads)
    assert np.array_equal(e, ref[0]) and np.array_equal(c, ref[1])
    # grid size with the floor-divided steps of Sec. 5 (rows x columns, plus
    # the last row and the last column); gamma_end adds one splitter
    si, sj = max(1, 300 // l), max(1, 250 // l)
    rows, cols = -(-300 // si), -(-250 // sj)
    assert 1 <= ni <= rows * cols + rows + cols


def test_alg1_int64_and_duplicates():
    rng = np.random.default_rng(21)
    fe, fc = random_poly(rng, 3, 200, 6, kind="i64")
    ge, gc = random_poly(rng, 3, 150, 6, kind="i64")
    ref = oracle.mul(3, [10] * 3, "i64", fe, fc, ge, gc)
    e, c, _ = oracle.mul_alg1(3, [10] * 3, "i64", fe, fc, ge, gc, l=5, threads=3)
    assert np.array_equal(e, ref[0]) and np.array_equal(c, ref[1])


def test_coef_at_matches_full_product():
    rng = np.random.default_rng(5)
    fe, fc = random_poly(rng, 3, 150, 6)
    ge, gc = random_poly(rng, 3, 120, 6)
    he, hc = oracle.mul(3, [10] * 3, "m61", fe, fc, ge, gc)
    got = oracle.coef_at(3, [10] * 3, "m61", fe, fc, ge, gc, he[::7])
    assert np.array_equal(got, hc[::7])
    absent = np.array([[13, 13, 13]], dtype=np.uint32)     # beyond the product's degree
    assert oracle.coef_at(3, [10] * 3, "m61", fe, fc, ge, gc, absent)[0] == 0


def test_paper_example1_operands():
    """Sec. 6, Example 1: f1 = (1+x+y+z+t)^40 has C(44, 4) = 135,751 terms,
    the count the paper prints; g1 = f1 + 1 differs only in the constant."""
    import math
    w = polygen.paper_example1()
    assert w.f.n == w.g.n == math.comb(44, 4) == 135751
    diff = np.flatnonzero(w.f.coefs != w.g.coefs)
    assert len(diff) == 1 and int(w.f.exps[diff[0]].sum()) == 0
    assert int(w.g.coefs[diff[0]]) == 2                 # 1 from the expansion, 1 added
    # x^40 has coefficient 1, x y z t^37 has 40!/37! = 59280
    row = {tuple(e): int(c) for e, c in zip(w.f.exps.tolist(), w.f.coefs.tolist())}
    assert row[(40, 0, 0, 0)] == 1 and row[(1, 1, 1, 37)] == 40 * 39 * 38


def test_eval_pow2_is_evaluation():
    """The power-of-two evaluation used on full-size results agrees with the
    oracle's plain evaluation (both mod 2^61 - 1)."""
    from tests.gpu_util import eval_pow2
    st = polygen.Stream(77, 0)
    e = st.below(200, 500 * 4).astype(np.uint32).reshape(500, 4)
    c = st.coef_m61(500)
    for a in ([1, 2, 3, 4], [60, 59, 7, 33], [0, 0, 0, 0]):
        assert eval_pow2(e, c, a) == oracle.evaluate(4, "m61", e, c, [pow(2, x, P61) for x in a])


def test_paper_examples_2_3_operands():
    """Sec. 6, Examples 2 and 3: the operands have C(30, 5) = 142,506 and
    C(33, 5) = 237,336 terms, the counts the paper prints."""
    for name, n in (("ex2", math.comb(30, 5)), ("ex3", math.comb(33, 5))):
        w = polygen.paper_example(name)
        assert w.f.n == w.g.n == n
    assert math.comb(30, 5) == 142506 and math.comb(33, 5) == 237336


# ---------------------------------------------------------------------------
# the exact-integer product (reference of the 192-bit kind)
# ---------------------------------------------------------------------------

def _from_words(c3):
    v = int(c3[0]) | (int(c3[1]) << 64) | (int(c3[2]) << 128)
    return v - (1 << 192) if v >> 191 else v


def test_exact_agrees_with_c_oracle_within_int128():
    """Two independent implementations (C with int128, Python integers)
    agree wherever int128 suffices."""
    st = polygen.Stream(91, 0)
    for nv, nf, ng in ((2, 40, 30), (3, 120, 90)):
        fe = st.below(6, nf * nv).astype(np.uint32).reshape(nf, nv)
        ge = st.below(6, ng * nv).astype(np.uint32).reshape(ng, nv)
        fc = st.coef_i64(nf, 1 << 40)
        gc = st.coef_i64(ng, 1 << 40)
        e1, c1 = oracle.mul(nv, [8] * nv, "i64", fe, fc, ge, gc)
        e2, c2 = oracle.mul_exact(nv, [8] * nv, fe, fc, ge, gc)
        np.testing.assert_array_equal(e1, e2)
        v1 = [int(c[0]) | (int(c[1]) << 64) for c in c1]
        v1 = [v - (1 << 128) if v >> 127 else v for v in v1]
        assert v1 == [_from_words(c) for c in c2]


def test_exact_closed_form_beyond_int128():
    """a (1 + x + ... + x^(n-1)) times b (1 + ... + x^(m-1)) with a, b near
    -2^63 and 2^63: the coefficient of x^k is a b times the number of pairs
    i + j = k, min(k + 1, n, m, n + m - 1 - k), up to 2^126 * 40 > 2^127."""
    a, b = -(2**63), 2**63 - 1
    n, m = 50, 40
    fe = np.arange(n, dtype=np.uint32).reshape(-1, 1)
    ge = np.arange(m, dtype=np.uint32).reshape(-1, 1)
    e, c = oracle.mul_exact(1, [16], fe, np.full(n, a, np.int64), ge, np.full(m, b, np.int64))
    assert e[:, 0].tolist() == list(range(n + m - 1))
    for k, ck in zip(e[:, 0].tolist(), c):
        assert _from_words(ck) == a * b * min(k + 1, n, m, n + m - 1 - k)
    assert max(abs(_from_words(ck)) for ck in c) > 2**127


def test_exact_brute_force_dense_convolution():
    """Tiny random cases with full-range int64 coefficients against a dense
    two-variable convolution in Python integers."""
    st = polygen.Stream(92, 0)
    for _ in range(3):
        fe = st.below(4, 10 * 2).astype(np.uint32).reshape(10, 2)
        ge = st.below(4, 8 * 2).astype(np.uint32).reshape(8, 2)
        fc = st.coef_i64(10, 2**62)
        gc = st.coef_i64(8, 2**62)
        A = [[0] * 4 for _ in range(4)]
        B = [[0] * 4 for _ in range(4)]
        for (x, y), v in zip(fe.tolist(), fc.tolist()):
            A[x][y] += v
        for (x, y), v in zip(ge.tolist(), gc.tolist()):
            B[x][y] += v
        H = {}
        for i in range(4):
            for j in range(4):
                for k in range(4):
                    for l in range(4):
                        if A[i][j] and B[k][l]:
                            H[(i + k, j + l)] = H.get((i + k, j + l), 0) + A[i][j] * B[k][l]
        want = sorted((k, v) for k, v in H.items() if v)
        e, c = oracle.mul_exact(2, [8, 8], fe, fc, ge, gc)
        assert [tuple(x) for x in e.tolist()] == [k for k, _ in want]
        assert [_from_words(x) for x in c] == [v for _, v in want]

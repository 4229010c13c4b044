"""Parity of the CUDA path with the oracle, through the C-ABI.

All coefficient arithmetic is exact, so the bar is bit-exact equality of keys
and coefficients.  Small and medium cases are compared element by element
with oracle.mul; the full-size workloads the benchmark times are checked on
sampled outputs (oracle.coef_at, one monomial at a time), by evaluation at
random points mod p (f(r) g(r) = h(r)) and by the closed-form term count.
"""

import math
import random

import numpy as np
import pytest

import oracle
import polygen
from tests.gpu_util import P61, assert_same, check_canonical, pack_np, run_gpu, unpack_np

pytestmark = pytest.mark.gpu

STRATS = [
    dict(strategy="auto"),
    dict(strategy="direct"),
    dict(strategy="direct", accumulator="wide"),
    dict(strategy="direct", accumulator="limbs", slots=2048),
    dict(strategy="direct", accumulator="limbs3", slots=3000),
    dict(strategy="direct", slots=512),            # many ranges, ragged tails
    dict(strategy="direct", slots=1000, ranges_per_sm=64),
    dict(strategy="direct", ranges_per_sm=3, cost_row=1, cost_window=1),   # other group boundaries
    dict(strategy="direct", grid_l=64),            # the paper's Sec. 5 grid for the group costs
    dict(strategy="sort"),
    dict(strategy="sort", grid_l=64),              # the paper's grid as the first splitters
    dict(strategy="sort", grid_l=1),
    dict(strategy="sort", chunk=256),              # single-monomial ranges above the chunk
    dict(strategy="sort", chunk=1000),
]


def _oracle(w, fe=None, fc=None, ge=None, gc=None):
    fe = w.f.exps if fe is None else fe
    fc = w.f.coefs if fc is None else fc
    ge = w.g.exps if ge is None else ge
    gc = w.g.coefs if gc is None else gc
    return oracle.mul(w.nvars, w.field_bits, w.kind, fe, fc, ge, gc)


@pytest.mark.parametrize("opts", STRATS, ids=lambda o: "-".join(f"{k}{v}" for k, v in o.items()))
def test_sparse4v_exact(opts):
    w = polygen.workload_sparse4v()
    ref = _oracle(w)
    gpu = run_gpu(w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs, **opts)
    check_canonical(gpu[0], gpu[1], w.field_bits)
    assert_same(gpu, ref, w.field_bits)
    assert gpu[2]["term_products"] == 10**6


@pytest.mark.parametrize("kind", ["m61", "i64"])
@pytest.mark.parametrize("opts", STRATS[:8], ids=lambda o: "-".join(f"{k}{v}" for k, v in o.items()))
def test_dense_reduced_exact(kind, opts):
    mons = polygen.monomials_total_degree(4, 10)          # 1001 monomials
    st = polygen.Stream(1234, 0)
    if kind == "m61":
        fc, gc = st.coef_m61(len(mons)), st.coef_m61(len(mons))
    else:
        fc, gc = st.coef_i64(len(mons), 1 << 20), st.coef_i64(len(mons), 1 << 20)
    ref = oracle.mul(4, [16] * 4, kind, mons, fc, mons[::-1], gc)
    gpu = run_gpu([16] * 4, kind, mons, fc, mons[::-1], gc, **opts)
    check_canonical(gpu[0], gpu[1], [16] * 4, kind)
    assert_same(gpu, (ref[0], ref[1].reshape(-1)), [16] * 4)
    assert len(ref[0]) == math.comb(4 + 20, 4)


def _sampled_check(w, gpu, nsample=120, seed=0):
    keys, coefs, _ = gpu
    kind = w.kind
    rnd = random.Random(seed)
    n = keys.shape[0]
    idx = sorted(rnd.sample(range(n), min(nsample, n)))
    exps = unpack_np(keys[idx], w.field_bits)
    want = oracle.coef_at(w.nvars, w.field_bits, kind, w.f.exps, w.f.coefs, w.g.exps, w.g.coefs, exps)
    got = coefs.reshape(n, -1)[idx]
    np.testing.assert_array_equal(got.reshape(want.shape), want)
    # evaluation at random points: h(r) = f(r) g(r) mod p
    for _ in range(2):
        r = [rnd.randrange(P61) for _ in range(w.nvars)]
        hk = "m61" if kind == "m61" else "i128"
        hv = oracle.evaluate(w.nvars, hk, unpack_np(keys, w.field_bits), coefs.reshape(n, -1) if kind != "m61" else coefs, r)
        fv = oracle.evaluate(w.nvars, kind, w.f.exps, w.f.coefs, r)
        gv = oracle.evaluate(w.nvars, kind, w.g.exps, w.g.coefs, r)
        assert hv == fv * gv % P61


@pytest.mark.parametrize("kind", ["m61", "i64"])
@pytest.mark.parametrize("acc", ["auto", "wide"])
def test_dense4v_full_size(kind, acc):
    """The dense workload at full size: 10626 x 10626 terms, exactly
    C(44, 4) = 135751 result terms, sampled coefficients, evaluation."""
    w = polygen.workload_dense4v(kind)
    gpu = run_gpu(w.field_bits, kind, w.f.exps, w.f.coefs, w.g.exps, w.g.coefs, accumulator=acc)
    check_canonical(gpu[0], gpu[1], w.field_bits, kind)
    assert gpu[0].shape[0] == math.comb(44, 4)
    assert gpu[2]["term_products"] == 10626 ** 2
    _sampled_check(w, gpu)


@pytest.mark.parametrize("nf,ng,slots", [(5000, 5000, 0), (3000, 2500, 1024), (2100, 40, 0)])
@pytest.mark.parametrize("kind", ["m61", "i64"])
def test_direct_every_row_has_products(nf, ng, slots, kind):
    """Univariate dense operands: every row that reaches a window has
    products in it, so a pass of the accumulate kernel finds more rows with
    products among its 2048 candidates than its 1024-row table holds and
    the next pass starts at the first row left out.  Ragged sizes, a small
    window and one short operand cover the pass ends."""
    st = polygen.Stream(4321, nf + ng)
    fe = np.arange(nf, dtype=np.uint32).reshape(-1, 1)
    ge = np.arange(ng, dtype=np.uint32)[::-1].copy().reshape(-1, 1)
    if kind == "m61":
        fc, gc = st.coef_m61(nf), st.coef_m61(ng)
    else:
        fc, gc = st.coef_i64(nf, 1 << 30), st.coef_i64(ng, 1 << 30)
    w = polygen.Workload("uni", 1, [16], kind, polygen.Poly(fe, fc), polygen.Poly(ge, gc))
    opts = dict(strategy="direct")
    if slots:
        opts["slots"] = slots
    gpu = run_gpu(w.field_bits, kind, fe, fc, ge, gc, **opts)
    assert gpu[2]["strategy"] == "direct"
    assert_same(gpu, _oracle(w), w.field_bits)


@pytest.mark.parametrize("acc", ["limbs3", "limbs", "wide"])
def test_direct_counters_at_their_bound(acc):
    """Every coefficient p - 1 or a value whose split form makes the largest
    limbs, univariate operands of 5000 terms: the middle slots receive
    5000 products each, over five passes of at most 1023 rows, so the
    three-limb counters reach their bound between normalisations."""
    nf = ng = 5000
    P61 = (1 << 61) - 1
    fe = np.arange(nf, dtype=np.uint32).reshape(-1, 1)
    ge = np.arange(ng, dtype=np.uint32)[::-1].copy().reshape(-1, 1)
    # the largest residues and the extreme 31-bit halves of the split form
    big = [P61 - 1, P61 - 2, (((1 << 30) - 1) << 31) + 5, (1 << 31) - 1]
    fc = np.array([big[i % 4] for i in range(nf)], dtype=np.uint64)
    gc = np.array([big[(i + 1) % 4] for i in range(ng)], dtype=np.uint64)
    w = polygen.Workload("uni_max", 1, [16], "m61", polygen.Poly(fe, fc), polygen.Poly(ge, gc))
    gpu = run_gpu(w.field_bits, "m61", fe, fc, ge, gc, strategy="direct", accumulator=acc)
    assert gpu[2]["strategy"] == "direct"
    assert_same(gpu, _oracle(w), w.field_bits)


def test_sparse5v_reduced_exact():
    w = polygen.workload_sparse5v(n=3000)
    ref = _oracle(w)
    for opts in (dict(strategy="auto"), dict(strategy="sort"), dict(strategy="direct", slots=4096),
                 dict(strategy="direct", accumulator="wide")):
        gpu = run_gpu(w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs, **opts)
        assert_same(gpu, ref, w.field_bits)


def test_sparse5v_full_size():
    """The sparse five-variable workload at full size (2.5e9 term products)."""
    w = polygen.workload_sparse5v()
    gpu = run_gpu(w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
    keys = gpu[0]
    check_canonical(keys, gpu[1], w.field_bits)
    assert keys.shape[0] <= 13 * 17 * 21 * 25 * 33
    _sampled_check(w, gpu, nsample=60)
    # monomials absent from the result have coefficient 0 in the oracle
    rnd = random.Random(3)
    box = [13, 17, 21, 25, 33]
    cand = np.array([[rnd.randrange(b) for b in box] for _ in range(400)], dtype=np.uint32)
    ck = pack_np(cand, w.field_bits)
    pos = np.minimum(np.searchsorted(keys, ck), keys.shape[0] - 1)
    absent = cand[keys[pos] != ck][:40]
    assert absent.shape[0] > 0
    z = oracle.coef_at(5, w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs, absent)
    assert np.all(z == 0)


@pytest.mark.parametrize("nv,nf,ng,seed", [(3, 16, 16, 1), (4, 700, 900, 2), (5, 100, 4096, 3),
                                           (8, 4096, 350, 4), (6, 2500, 2500, 5), (3, 1, 4000, 6)])
def test_sparse_exact(nv, nf, ng, seed):
    w = polygen.sparse_product(polygen.Stream(seed, 0), nv, nf, ng)
    ref = _oracle(w)
    for opts in (dict(strategy="auto"), dict(strategy="sort", chunk=512)):
        gpu = run_gpu(w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs, **opts)
        check_canonical(gpu[0], gpu[1], w.field_bits)
        assert_same(gpu, ref, w.field_bits)


def test_sparse_heavy_collisions():
    """Sparse supports with a small exponent cap: many products per monomial."""
    w = polygen.sparse_product(polygen.Stream(77, 0), 4, 3000, 3000, exp_hi=7)
    ref = _oracle(w)
    for opts in (dict(strategy="auto"), dict(strategy="sort", chunk=300), dict(strategy="direct", slots=64)):
        gpu = run_gpu(w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs, **opts)
        assert_same(gpu, ref, w.field_bits)


def test_commutative_bit_exact():
    w = polygen.workload_sparse4v()
    a = run_gpu(w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
    b = run_gpu(w.field_bits, "m61", w.g.exps, w.g.coefs, w.f.exps, w.f.coefs)
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])


def test_power_closed_form():
    """(1+x+y+z)^6 (1+x+y+z)^7 = (1+x+y+z)^13, multinomial coefficients."""
    fe, fc = polygen.multinomial_power(3, 6)
    ge, gc = polygen.multinomial_power(3, 7)
    he, hc = polygen.multinomial_power(3, 13)
    for s in ("direct", "sort"):
        gpu = run_gpu([10] * 3, "m61", fe, np.array(fc, np.uint64), ge, np.array(gc, np.uint64), strategy=s)
        order = np.lexsort(he.T[::-1])
        np.testing.assert_array_equal(gpu[0], pack_np(he[order], [10] * 3))
        np.testing.assert_array_equal(gpu[1], np.array(hc, np.uint64)[order])


# ---------------------------------------------------------------------------
# edge cases and error rules
# ---------------------------------------------------------------------------

def test_empty_and_zero_operands():
    import paper_1303_7425_gb300 as P
    e = np.zeros((0, 3), np.uint32)
    c = np.zeros(0, np.uint64)
    fe = np.array([[1, 2, 3], [0, 0, 1]], np.uint32)
    k, co, st = run_gpu([8] * 3, "m61", fe, np.array([5, 7], np.uint64), e, c)
    assert k.shape == (0,)
    k, co, st = run_gpu([8] * 3, "m61", fe, np.array([0, P61], np.uint64), fe, np.array([1, 2], np.uint64))
    assert k.shape == (0,)


def test_duplicates_unsorted_and_unreduced_inputs():
    rng = np.random.default_rng(5)
    fe = rng.integers(0, 5, size=(400, 3)).astype(np.uint32)     # many repeats
    ge = rng.integers(0, 5, size=(300, 3)).astype(np.uint32)
    fc = rng.integers(0, 2**63, size=400, dtype=np.uint64) * np.uint64(2) + np.uint64(1)  # >= p too
    gc = rng.integers(0, 2**63, size=300, dtype=np.uint64)
    ref = oracle.mul(3, [8] * 3, "m61", fe, fc, ge, gc)
    for s in ("direct", "sort"):
        assert_same(run_gpu([8] * 3, "m61", fe, fc, ge, gc, strategy=s), ref, [8] * 3)


@pytest.mark.parametrize("bits,hi", [([32, 32], (1 << 30) - 1), ([4] * 16, 3), ([1, 31, 32], 1 << 29),
                                      ([20, 20, 20], (1 << 18) - 1)])
def test_packing_extremes(bits, hi):
    nv = len(bits)
    st = polygen.Stream(11, nv)
    lim = [min(hi, (1 << (b - 2)) - 1) if b >= 2 else 0 for b in bits]
    fe = np.stack([st.below(l + 1, 300).astype(np.uint32) for l in lim], axis=1)
    ge = np.stack([st.below(l + 1, 200).astype(np.uint32) for l in lim], axis=1)
    fe[0] = lim
    ge[0] = lim                                        # the largest exponent sum is reached
    fc, gc = st.coef_m61(300), st.coef_m61(200)
    ref = oracle.mul(nv, bits, "m61", fe, fc, ge, gc)
    for s in ("auto", "sort"):
        gpu = run_gpu(bits, "m61", fe, fc, ge, gc, strategy=s)
        assert_same(gpu, ref, bits)


@pytest.mark.parametrize("bits,lims", [([32], [(1 << 30) - 1]),            # extent 2^31 - 1
                                       ([16, 16], [(1 << 14) - 1, 3]),       # extents 2^15 - 1 and 7
                                       ([8, 8, 8, 8], [2, 63, 1, 40])])      # small odd extents
def test_direct_rank_decoding_extents(bits, lims):
    """Forced direct strategy on boxes whose extents run from 3 to 2^31 - 1:
    every output key is rebuilt from its rank by division by the extents."""
    nv = len(bits)
    st = polygen.Stream(17, nv)
    fe = np.stack([st.below(l + 1, 40).astype(np.uint32) for l in lims], axis=1)
    ge = np.stack([st.below(l + 1, 30).astype(np.uint32) for l in lims], axis=1)
    fe[0] = lims
    ge[0] = lims                                        # the largest exponent sum is reached
    fc, gc = st.coef_m61(40), st.coef_m61(30)
    ref = oracle.mul(nv, bits, "m61", fe, fc, ge, gc)
    gpu = run_gpu(bits, "m61", fe, fc, ge, gc, strategy="direct")
    assert gpu[2]["strategy"] == "direct"
    assert_same(gpu, ref, bits)


@pytest.mark.parametrize("case", ["sparse4v", "dense_i64", "sparse3", "sparse5", "collisions"])
def test_hash_strategy_exact(case):
    """Hashed windows (PM_STRATEGY_HASH) on dense, sparse and colliding
    products, both coefficient kinds: bit-exact with the oracle."""
    if case == "sparse4v":
        w = polygen.workload_sparse4v()
    elif case == "dense_i64":
        mons = polygen.monomials_total_degree(3, 10)
        st = polygen.Stream(5, 1)
        w = polygen.Workload("d3", 3, [12] * 3, "i64", polygen.Poly(mons, st.coef_i64(len(mons), 1 << 40)),
                             polygen.Poly(mons[::-1].copy(), st.coef_i64(len(mons), 1 << 40)))
    elif case == "sparse3":
        w = polygen.sparse_product(polygen.Stream(8, 0), 3, 700, 500, 200)
    elif case == "sparse5":
        w = polygen.sparse_product(polygen.Stream(9, 0), 5, 1500, 900, 30)
    else:
        st = polygen.Stream(10, 0)
        e = st.below(6, 800 * 3).astype(np.uint32).reshape(800, 3)
        w = polygen.Workload("col", 3, [10] * 3, "m61", polygen.Poly(e, st.coef_m61(800)),
                             polygen.Poly(e[::-1].copy(), st.coef_m61(800)))
    ref = _oracle(w)
    gpu = run_gpu(w.field_bits, w.kind, w.f.exps, w.f.coefs, w.g.exps, w.g.coefs, strategy="hash")
    assert gpu[2]["strategy"] == "hash"
    assert_same(gpu, ref, w.field_bits)


@pytest.mark.parametrize("case", ["sparse5", "colliding"])
def test_hash_wide_accumulator_exact(case):
    """Hashed windows with the wide accumulator asked for (a 64-bit sum and
    its wrap count per slot, the one the library picks for operands above
    65537 terms, whose windows otherwise switch to the limbs): bit-exact
    with the oracle, also over the splits of overflowing windows."""
    if case == "sparse5":
        w = polygen.sparse_product(polygen.Stream(9, 0), 5, 1500, 900, 30)
    else:
        w = polygen.sparse_product(polygen.Stream(12, 0), 3, 2000, 2000, 400)
    ref = _oracle(w)
    gpu = run_gpu(w.field_bits, w.kind, w.f.exps, w.f.coefs, w.g.exps, w.g.coefs, strategy="hash",
                  accumulator="wide")
    assert gpu[2]["strategy"] == "hash"
    assert_same(gpu, ref, w.field_bits)


def test_hash_windows_split_when_full():
    """4 million term products, nearly all distinct, over a box of 5e8 ranks:
    the first windows (about 6,600 monomials each) overflow their tables,
    are split over several rounds, and the result is still exact."""
    w = polygen.sparse_product(polygen.Stream(12, 0), 3, 2000, 2000, 400)
    ref = _oracle(w)
    gpu = run_gpu(w.field_bits, w.kind, w.f.exps, w.f.coefs, w.g.exps, w.g.coefs, strategy="hash")
    assert gpu[2]["refine_rounds"] >= 2
    assert_same(gpu, ref, w.field_bits)


@pytest.mark.parametrize("strategy", ["direct", "sort", "hash"])
def test_int192_exact_beyond_int128(strategy):
    """int64 coefficients up to 2^62 in magnitude with up to ~40 products per
    result monomial: sums beyond 2^127, which the 128-bit kind refuses
    (PM_ECOEF_BOUND) and the 192-bit kind computes exactly, compared with
    the exact-integer oracle."""
    import paper_1303_7425_gb300 as P
    st = polygen.Stream(33, 0)
    mons = polygen.monomials_total_degree(3, 6)                 # 84 monomials
    fe = np.concatenate([mons, st.below(7, 200 * 3).astype(np.uint32).reshape(200, 3)])
    ge = np.concatenate([mons[::-1], st.below(7, 150 * 3).astype(np.uint32).reshape(150, 3)])
    fc = st.coef_i64(len(fe), 2**62)
    gc = st.coef_i64(len(ge), 2**62)
    fc[0] = gc[0] = -(2**62)
    bits = [10, 10, 10]
    # repeated monomials are summed on load: keep every combined value in int64
    fe, fc = _combine_in_int64(fe, fc)
    ge, gc = _combine_in_int64(ge, gc)
    e, c = oracle.mul_exact(3, bits, fe, fc, ge, gc)
    vals = [int(x[0]) | (int(x[1]) << 64) | (int(x[2]) << 128) for x in c]
    assert any(abs(v - (1 << 192) if v >> 191 else v) >= 2**127 for v in vals)
    with pytest.raises(P.PolymulError) as ei:
        run_gpu(bits, "i64", fe, fc, ge, gc, strategy=strategy)
    assert ei.value.code == -3
    gpu = run_gpu(bits, "i192", fe, fc, ge, gc, strategy=strategy)
    assert gpu[2]["strategy"] == strategy
    assert_same(gpu, (e, c), bits)


def _combine_in_int64(e, c):
    """Merge repeated exponent rows, keeping each sum inside int64 by
    dropping the repeats that would leave it."""
    seen = {}
    for row, v in zip(map(tuple, e.tolist()), c.tolist()):
        s = seen.get(row, 0) + int(v)
        if -2**63 <= s < 2**63 and s != 0:
            seen[row] = s
    rows = list(seen)
    return np.array(rows, dtype=np.uint32), np.array([seen[r] for r in rows], dtype=np.int64)


def test_int128_near_bound():
    a, b = -2**63, 2**63 - 1
    fe = np.array([[0], [1]], np.uint32)
    ref = oracle.mul(1, [8], "i64", fe, np.array([a, a], np.int64), fe, np.array([b, b], np.int64))
    for s in ("direct", "sort"):
        gpu = run_gpu([8], "i64", fe, np.array([a, a], np.int64), fe, np.array([b, b], np.int64), strategy=s)
        assert_same(gpu, (ref[0], ref[1].reshape(-1)), [8])


def _expect_error(code, *args, **kw):
    import paper_1303_7425_gb300 as P
    with pytest.raises(P.PolymulError) as ei:
        run_gpu(*args, **kw)
    assert ei.value.code == code
    return ei.value


def test_error_rules():
    one = np.array([1], np.uint64)
    _expect_error(-2, [4, 4], "m61", np.array([[8, 0]], np.uint32), one, np.array([[0, 0]], np.uint32), one)
    _expect_error(-2, [4, 4], "m61", np.array([[4, 0]], np.uint32), one, np.array([[4, 0]], np.uint32), one)
    fe = np.array([[0], [1]], np.uint32)
    _expect_error(-3, [8], "i64", fe, np.array([-2**63, -2**63], np.int64), fe, np.array([-2**63, 1], np.int64))
    _expect_error(-3, [8], "i64", np.array([[0], [0]], np.uint32), np.array([2**62, 2**62], np.int64),
                  fe, np.array([1, 1], np.int64))
    _expect_error(-1, [40, 30], "m61", fe.repeat(2, 1), np.array([1, 2], np.uint64), fe.repeat(2, 1),
                  np.array([1, 2], np.uint64))


def test_capacity_error_reports_needed_size():
    import paper_1303_7425_gb300 as P
    import torch
    from tests.gpu_util import to_dev
    w = polygen.workload_sparse4v()
    f = to_dev(w.f.exps, w.f.coefs)
    g = to_dev(w.g.exps, w.g.coefs)
    out = (torch.empty(10, dtype=torch.int64, device="cuda"), torch.empty(10, dtype=torch.int64, device="cuda"))
    with pytest.raises(P.PolymulError) as ei:
        P.polymul(w.field_bits, f[0], f[1], g[0], g[1], out=out)
    assert ei.value.code == -4
    ref = _oracle(w)
    assert ei.value.needed == len(ref[0])


def test_pack_unpack_roundtrip():
    import paper_1303_7425_gb300 as P
    import torch
    bits = [7, 9, 11, 5]
    st = polygen.Stream(3, 3)
    e = np.stack([st.below(1 << (b - 1), 1000).astype(np.uint32) for b in bits], axis=1)
    de = torch.from_numpy(e.view(np.int32)).cuda()
    keys = P.pack(bits, de)
    np.testing.assert_array_equal(keys.cpu().numpy().view(np.uint64), pack_np(e, bits))
    back = P.unpack(bits, keys)
    np.testing.assert_array_equal(back.cpu().numpy().view(np.uint32), e)


@pytest.mark.parametrize("case", ["sparse5", "sparse3", "sparse8", "i64", "dense_collisions", "hot_keys"])
def test_bucket_strategy_exact(case):
    """The bucketed strategy (every term product to a bucket of its key,
    buckets sorted in shared memory; buckets above the chunk by a device-wide
    sort): bit-exact with the oracle on sparse products, int64 inputs, dense
    operands whose products collide on every key, and univariate operands
    whose middle keys draw more products than a bucket holds."""
    if case == "sparse5":
        w = polygen.sparse_product(polygen.Stream(51, 0), 5, 1500, 900)
    elif case == "sparse3":
        w = polygen.sparse_product(polygen.Stream(52, 0), 3, 2000, 1700, 300)
    elif case == "sparse8":
        w = polygen.sparse_product(polygen.Stream(53, 0), 8, 700, 3000)
    elif case == "i64":
        st = polygen.Stream(54, 0)
        e = polygen.distinct_random_vectors(st, 1200, 4, 4000)
        g = polygen.distinct_random_vectors(st, 1100, 4, 4000)
        w = polygen.Workload("b64", 4, [16] * 4, "i64", polygen.Poly(e, st.coef_i64(1200, 1 << 40)),
                             polygen.Poly(g, st.coef_i64(1100, 1 << 40)))
    elif case == "dense_collisions":
        mons = polygen.monomials_total_degree(3, 14)
        st = polygen.Stream(55, 0)
        w = polygen.Workload("bd", 3, [12] * 3, "m61", polygen.Poly(mons, st.coef_m61(len(mons))),
                             polygen.Poly(mons[::-1].copy(), st.coef_m61(len(mons))))
    else:
        st = polygen.Stream(56, 0)
        fe = np.arange(4300, dtype=np.uint32).reshape(-1, 1)
        w = polygen.Workload("hot", 1, [16], "m61", polygen.Poly(fe, st.coef_m61(4300)),
                             polygen.Poly(fe[::-1].copy(), st.coef_m61(4300)))
    ref = _oracle(w)
    gpu = run_gpu(w.field_bits, w.kind, w.f.exps, w.f.coefs, w.g.exps, w.g.coefs, strategy="bucket")
    assert gpu[2]["strategy"] == "bucket"
    if case == "hot_keys":
        assert gpu[2]["refine_rounds"] > 0          # buckets sorted outside shared memory
    assert_same(gpu, ref, w.field_bits)


def test_bucket_strategy_chosen_for_large_sparse_products():
    """Sparse products of at least 2^20 term products whose result box is
    more than 64 times the work take the bucketed strategy by default, and
    give the sort strategy's result bit for bit."""
    import paper_1303_7425_gb300 as P
    w = polygen.sparse_product(polygen.Stream(57, 0), 5, 1500, 1200)
    gpu = run_gpu(w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
    assert gpu[2]["strategy"] == "bucket"
    srt = run_gpu(w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs, strategy="sort")
    np.testing.assert_array_equal(gpu[0], srt[0])
    np.testing.assert_array_equal(gpu[1], srt[1])
    with pytest.raises(P.PolymulError) as ei:                       # no 192-bit bucket path
        run_gpu(w.field_bits, "i192", w.f.exps, w.f.coefs.astype(np.int64) >> 4, w.g.exps,
                w.g.coefs.astype(np.int64) >> 4, strategy="bucket")
    assert ei.value.code == -1

"""The batched pass (pm_batch_*): every product of a mixed batch equals the
oracle and equals the same product computed alone by pm_polymul (bit-exact),
errors stay per item, and replaying the captured graph recomputes from the
current inputs."""

import numpy as np
import pytest

import oracle
import polygen
from tests.gpu_util import pack_np, to_dev

pytestmark = pytest.mark.gpu


def _product(w, cap=None):
    import torch
    f = to_dev(w.f.exps, w.f.coefs, w.kind)
    g = to_dev(w.g.exps, w.g.coefs, w.kind)
    cap = cap if cap is not None else max(w.f.n * w.g.n, 1)
    words = 1 if w.kind == "m61" else 2
    out = (torch.full((cap,), -1, dtype=torch.int64, device="cuda"),
           torch.full((cap, words) if words == 2 else (cap,), -1, dtype=torch.int64, device="cuda"))
    return dict(field_bits=w.field_bits, kind=w.kind, f_exps=f[0], f_coefs=f[1], g_exps=g[0], g_coefs=g[1],
                out=out, w=w)


def _mixed_workloads(seed=5, count=40):
    st = polygen.Stream(seed, 0)
    ws = []
    nv = 3 + st.below(6, count).astype(int)
    nf = polygen.log_uniform_size(st, count, 16, 1200)
    ng = polygen.log_uniform_size(st, count, 16, 1200)
    for k in range(count):
        ws.append(polygen.sparse_product(polygen.Stream(seed, 100 + k), int(nv[k]), int(nf[k]), int(ng[k])))
    # dense small products (many products per monomial)
    mons = polygen.monomials_total_degree(3, 8)
    s2 = polygen.Stream(seed, 999)
    ws.append(polygen.Workload("dense3", 3, [10] * 3, "m61", polygen.Poly(mons, s2.coef_m61(len(mons))),
                               polygen.Poly(mons[::-1].copy(), s2.coef_m61(len(mons)))))
    # int64 kind with repeated monomials
    e = s2.below(4, 300 * 3).astype(np.uint32).reshape(300, 3)
    ws.append(polygen.Workload("i64rep", 3, [8] * 3, "i64", polygen.Poly(e, s2.coef_i64(300, 1 << 30)),
                               polygen.Poly(e[::-1].copy(), s2.coef_i64(300, 1 << 30))))
    return ws


def _check_against_oracle(pr, n):
    w = pr["w"]
    e, c = oracle.mul(w.nvars, w.field_bits, w.kind, w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
    assert n == len(e)
    keys = pr["out"][0][:n].cpu().numpy().view(np.uint64)
    coefs = pr["out"][1][:n].cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(keys, pack_np(e, w.field_bits))
    np.testing.assert_array_equal(coefs.reshape(-1), np.asarray(c, dtype=np.uint64).reshape(-1))


@pytest.mark.parametrize("opts", [dict(), dict(range_target=64, ranges_per_item=1), dict(range_target=3072,
                                                                                          ranges_per_item=64)])
def test_batch_matches_oracle_and_single(opts):
    import paper_1303_7425_gb300 as P
    prods = [_product(w) for w in _mixed_workloads()]
    res, stats = P.batch_polymul(prods, **opts)
    assert stats["graph"] == 1
    for pr, (status, n) in zip(prods, res):
        assert status == 0
        _check_against_oracle(pr, n)
        single = P.polymul(pr["field_bits"], pr["f_exps"], pr["f_coefs"], pr["g_exps"], pr["g_coefs"], kind=pr["kind"])
        assert single.n == n
        np.testing.assert_array_equal(single.keys.cpu().numpy(), pr["out"][0][:n].cpu().numpy())
        np.testing.assert_array_equal(single.coefs.cpu().numpy(), pr["out"][1][:n].cpu().numpy())


@pytest.mark.parametrize("opts", [dict(), dict(range_target=4096, ranges_per_item=64),
                                  dict(range_target=100, ranges_per_item=3)])
def test_batch_mod_p_only_wider_chunk(opts):
    """A batch whose products are all mod p keeps one coefficient word per
    product in shared memory and sorts up to 4096 products per piece; ranges
    up to that size (and the bisection above it) stay exact."""
    import paper_1303_7425_gb300 as P
    ws = [w for w in _mixed_workloads(seed=17, count=24) if w.kind == "m61"]
    prods = [_product(w) for w in ws]
    res, stats = P.batch_polymul(prods, **opts)
    assert stats["graph"] == 1
    for pr, (status, n) in zip(prods, res):
        assert status == 0
        _check_against_oracle(pr, n)


def test_batch_range_target_limit_depends_on_kinds():
    """4096 products per range fit only one coefficient word per product: with
    an int64 item in the batch the same option is rejected."""
    import paper_1303_7425_gb300 as P
    ws = _mixed_workloads(seed=19, count=3)
    assert any(w.kind == "i64" for w in ws)
    with pytest.raises(P.PolymulError) as ei:
        P.batch_polymul([_product(w) for w in ws], range_target=4096)
    assert ei.value.code == -1
    res, _ = P.batch_polymul([_product(w) for w in ws], range_target=3072)
    assert all(st == 0 for st, _ in res)


def test_batch_errors_stay_per_item():
    import paper_1303_7425_gb300 as P
    ws = _mixed_workloads(count=6)
    prods = [_product(w) for w in ws]
    one = np.array([1], np.uint64)
    bad = polygen.Workload("ovf", 2, [4, 4], "m61", polygen.Poly(np.array([[4, 0]], np.uint32), one),
                           polygen.Poly(np.array([[4, 1]], np.uint32), one))
    small = _product(ws[0], cap=3)
    zero = polygen.Workload("zero", 2, [8, 8], "m61", polygen.Poly(np.array([[1, 1], [2, 2]], np.uint32),
                                                                   np.array([0, 0], np.uint64)),
                            polygen.Poly(np.array([[1, 0]], np.uint32), one))
    prods = prods[:3] + [_product(bad), small, _product(zero)] + prods[3:]
    res, _ = P.batch_polymul(prods)
    for k, (pr, (status, n)) in enumerate(zip(prods, res)):
        if k == 3:
            assert status == -2
        elif k == 4:
            assert status == -4 and n > 3
        elif k == 5:
            assert status == 0 and n == 0
        else:
            assert status == 0
            _check_against_oracle(pr, n)


def test_batch_heavy_multiplicity():
    """Univariate dense operands: up to 3500 products per monomial, so ranges
    above the shared-memory chunk are bisected and single monomials summed."""
    import paper_1303_7425_gb300 as P
    st = polygen.Stream(31, 0)
    e = np.arange(3500, dtype=np.uint32).reshape(-1, 1)
    w = polygen.Workload("uni", 1, [16], "m61", polygen.Poly(e, st.coef_m61(3500)),
                         polygen.Poly(e[::-1].copy(), st.coef_m61(3500)))
    prods = [_product(w, cap=7000)]
    res, stats = P.batch_polymul(prods)
    assert res[0][0] == 0
    _check_against_oracle(prods[0], res[0][1])


@pytest.mark.parametrize("opts", [dict(), dict(range_target=64, ranges_per_item=1)])
def test_direct_and_copied_outputs_agree(opts):
    """The same products twice in one batch: once with h.cap >= n_f n_g
    (ranges written straight into h, moved left where monomials repeat) and
    once with h.cap equal to the result's size (ranges copied in from the
    workspace).  Both equal the oracle; the univariate dense product makes
    up to 900 term products per monomial, so nearly every range moves."""
    import paper_1303_7425_gb300 as P
    st = polygen.Stream(41, 0)
    e = np.arange(900, dtype=np.uint32).reshape(-1, 1)
    uni = polygen.Workload("uni", 1, [16], "m61", polygen.Poly(e, st.coef_m61(900)),
                           polygen.Poly(e[::-1].copy(), st.coef_m61(900)))
    ws = [uni] + _mixed_workloads(seed=17, count=8)
    exact = []
    for w in ws:
        ex, _ = oracle.mul(w.nvars, w.field_bits, w.kind, w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
        exact.append(max(len(ex), 1))
    direct = [_product(w) for w in ws]
    copied = [_product(w, cap=n) for w, n in zip(ws, exact)]
    res, stats = P.batch_polymul(direct + copied, **opts)
    assert stats["term_products"] == 2 * sum(w.f.n * w.g.n for w in ws)
    for pr, (status, n) in zip(direct + copied, res):
        assert status == 0
        _check_against_oracle(pr, n)


@pytest.mark.parametrize("kind", ["m61", "i64"])
def test_direct_outputs_moved_by_many_units(kind):
    """A large sparse product with two repeated monomials near the bottom of
    the key order: nearly its whole output moves left by one or two terms,
    unit after unit, each unit's destination overlapping the sources of the
    one before it.  Small ranges make each unit span several."""
    import paper_1303_7425_gb300 as P
    base = polygen.sparse_product(polygen.Stream(57, 0), 3, 2500, 2400)
    fe, ge = base.f.exps.copy(), base.g.exps.copy()
    # x^0 and x_3 in both operands: x_3 arises twice; x_2 x_3 likewise
    fe[0], fe[1], fe[2] = (0, 0, 0), (0, 0, 1), (0, 1, 0)
    ge[0], ge[1], ge[2] = (0, 0, 0), (0, 0, 1), (0, 1, 1)
    assert len({tuple(r) for r in fe}) == len(fe) and len({tuple(r) for r in ge}) == len(ge)
    st = polygen.Stream(58, 0)
    if kind == "m61":
        fc, gc = st.coef_m61(len(fe)), st.coef_m61(len(ge))
    else:
        fc, gc = st.coef_i64(len(fe), 1 << 40), st.coef_i64(len(ge), 1 << 40)
    w = polygen.Workload("moves", 3, base.field_bits, kind, polygen.Poly(fe, fc), polygen.Poly(ge, gc))
    e, c = oracle.mul(w.nvars, w.field_bits, w.kind, w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
    keys, coefs = pack_np(e, w.field_bits), np.asarray(c, dtype=np.uint64).reshape(-1)
    assert len(e) == w.f.n * w.g.n - 2
    for opts in (dict(range_target=64, ranges_per_item=4), dict()):
        prods = [_product(w)]
        res, stats = P.batch_polymul(prods, **opts)
        assert res[0] == (0, len(e))
        np.testing.assert_array_equal(prods[0]["out"][0][:len(e)].cpu().numpy().view(np.uint64), keys)
        np.testing.assert_array_equal(prods[0]["out"][1][:len(e)].cpu().numpy().view(np.uint64).reshape(-1), coefs)


@pytest.mark.parametrize("kind", ["m61", "i64"])
def test_batch_clustered_keys_take_the_radix_path(kind):
    """Keys clustered inside a range's interval (64 x 64 products packed in a
    small corner of a span of about 2^52) put more than 32 pairs into one
    bucket, so the range kernel sorts those pieces by radix instead; one far
    term of f stretches the span.  The result must still equal the oracle."""
    import paper_1303_7425_gb300 as P
    i = np.arange(64, dtype=np.uint32)
    fe = np.stack([np.concatenate([i, [1 << 20]]), np.zeros(65, np.uint32)], axis=1).astype(np.uint32)
    ge = np.stack([np.zeros(64, np.uint32), i], axis=1).astype(np.uint32)
    st = polygen.Stream(77, 0)
    if kind == "m61":
        fc, gc = st.coef_m61(65), st.coef_m61(64)
    else:
        fc, gc = st.coef_i64(65, 1 << 40), st.coef_i64(64, 1 << 40)
    w = polygen.Workload("cluster", 2, [32, 32], kind, polygen.Poly(fe, fc), polygen.Poly(ge, gc))
    for opts in (dict(), dict(range_target=1024, ranges_per_item=2)):
        prods = [_product(w)]
        res, _ = P.batch_polymul(prods, **opts)
        assert res[0][0] == 0
        _check_against_oracle(prods[0], res[0][1])


@pytest.mark.parametrize("kind", ["m61", "i64"])
def test_batch_operands_above_4096_terms(kind):
    """An operand above 4096 terms switches the range kernel to its layout
    for up to PM_BATCH_MAX_TERMS terms; the small products beside it must
    come out the same."""
    import paper_1303_7425_gb300 as P
    st = polygen.Stream(88, 0)
    big = polygen.sparse_product(polygen.Stream(88, 1), 3, 6000, 40)
    big.f.coefs = st.coef_m61(6000) if kind == "m61" else st.coef_i64(6000, 1 << 30)
    big.g.coefs = st.coef_m61(40) if kind == "m61" else st.coef_i64(40, 1 << 30)
    big.kind = kind
    ws = [big] + [w for w in _mixed_workloads(seed=23, count=6) if w.kind == "m61"]
    prods = [_product(w) for w in ws]
    res, _ = P.batch_polymul(prods)
    for pr, (status, n) in zip(prods, res):
        assert status == 0
        _check_against_oracle(pr, n)


def test_graph_replay_recomputes_from_inputs():
    import paper_1303_7425_gb300 as P
    ws = _mixed_workloads(seed=9, count=12)
    prods = [_product(w) for w in ws]
    plan = P.BatchPlan(prods)
    try:
        plan.run()
        res1, _ = plan.finish()
        for pr, (status, n) in zip(prods, res1):
            assert status == 0
            _check_against_oracle(pr, n)
        # change product 0's coefficients in place and replay
        w0 = ws[0]
        new = polygen.Stream(123, 0).coef_m61(w0.f.n)
        prods[0]["f_coefs"].copy_(to_dev(w0.f.exps, new)[1])
        w0.f.coefs = new
        plan.run()
        plan.run()
        res2, _ = plan.finish()
        for pr, (status, n) in zip(prods, res2):
            assert status == 0
            _check_against_oracle(pr, n)
    finally:
        plan.close()

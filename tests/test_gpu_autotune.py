"""The autotuner: it times every candidate on the product, keeps the fastest
for the shape class, and pm_polymul with default options then uses that
choice; the result is bit-exact whatever configuration runs."""

import numpy as np
import pytest

import oracle
import polygen
from tests.gpu_util import assert_same, to_dev

pytestmark = pytest.mark.gpu


def test_autotune_then_default_call_uses_it():
    import paper_1303_7425_gb300 as P
    w = polygen.workload_sparse4v()
    f = to_dev(w.f.exps, w.f.coefs)
    g = to_dev(w.g.exps, w.g.coefs)
    best, table = P.autotune(w.field_bits, f[0], f[1], g[0], g[1])
    assert len(table) >= 8 and any(ms > 0 for _, ms in table)
    assert min(ms for _, ms in table if ms > 0) == pytest.approx(dict((str(o), ms) for o, ms in table)[str(best)])
    r = P.polymul(w.field_bits, f[0], f[1], g[0], g[1])
    assert r.stats["strategy"] == best["strategy"]
    ref = oracle.mul(w.nvars, w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
    assert_same((r.keys.cpu().numpy().view(np.uint64), r.coefs.cpu().numpy().view(np.uint64), None), ref,
                w.field_bits)


def test_autotune_sparse_refuses_direct_and_picks_sort():
    import paper_1303_7425_gb300 as P
    w = polygen.sparse_product(polygen.Stream(4, 0), 6, 1500, 900)
    f = to_dev(w.f.exps, w.f.coefs)
    g = to_dev(w.g.exps, w.g.coefs)
    best, table = P.autotune(w.field_bits, f[0], f[1], g[0], g[1])
    assert best["strategy"] == "sort"
    assert all(ms < 0 for o, ms in table if o["strategy"] == "direct")   # the box is far too large


def test_batch_autotune_returns_a_candidate():
    import torch

    import paper_1303_7425_gb300 as P
    ws = [polygen.sparse_product(polygen.Stream(8, k), 4, 200 + 10 * k, 300) for k in range(20)]
    prods = []
    for w in ws:
        f = to_dev(w.f.exps, w.f.coefs)
        g = to_dev(w.g.exps, w.g.coefs)
        cap = w.f.n * w.g.n
        prods.append(dict(field_bits=w.field_bits, f_exps=f[0], f_coefs=f[1], g_exps=g[0], g_coefs=g[1],
                          out=(torch.empty(cap, dtype=torch.int64, device="cuda"),
                               torch.empty(cap, dtype=torch.int64, device="cuda"))))
    best, table = P.batch_autotune(prods)
    assert best in [c for c, _ in table]
    res, _ = P.batch_polymul(prods, **best)
    assert all(s == 0 for s, _ in res)

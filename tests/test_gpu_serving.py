"""The serving engine: Poisson arrivals, continuous batching over several
streams, HBM-budget admission.  Each result must be the same in the mix as
alone (bit-exact, the tolerance of every test here), and equal the oracle."""

import numpy as np
import pytest

import oracle
import polygen
from tests.gpu_util import pack_np, to_dev

pytestmark = pytest.mark.gpu


def _prod(w):
    import torch
    f = to_dev(w.f.exps, w.f.coefs, w.kind)
    g = to_dev(w.g.exps, w.g.coefs, w.kind)
    cap = max(w.f.n * w.g.n, 1)
    if w.f.n > 8192 or w.g.n > 8192:          # dense products: their box bounds the result
        cap = 200_000
    out = (torch.full((cap,), -1, dtype=torch.int64, device="cuda"),
           torch.full((cap,), -1, dtype=torch.int64, device="cuda"))
    return dict(field_bits=w.field_bits, kind=w.kind, f_exps=f[0], f_coefs=f[1], g_exps=g[0], g_coefs=g[1],
                out=out)


def _stream(count=150, dense=3, seed=17, rate=20000.0, hi=800):
    st = polygen.Stream(seed, 0)
    nv = 3 + st.below(6, count).astype(int)
    nf = polygen.log_uniform_size(st, count, 16, hi)
    ng = polygen.log_uniform_size(st, count, 16, hi)
    ws = [polygen.sparse_product(polygen.Stream(seed, 10 + k), int(nv[k]), int(nf[k]), int(ng[k]))
          for k in range(count)]
    for k in range(dense):
        ws.insert(10 + 40 * k, polygen.workload_dense4v(seed=seed + k))
    gaps = -np.log(1.0 - st.uniform01(len(ws))) / rate
    return ws, np.cumsum(gaps)


def test_serving_results_equal_alone_and_oracle():
    import paper_1303_7425_gb300 as P
    from paper_1303_7425_gb300.serving import serve
    ws, t = _stream()
    prods = [_prod(w) for w in ws]
    rep = serve(list(zip(t.tolist(), prods)), [w.term_products for w in ws],
                server_kwargs=dict(streams=4, max_batch=16, device_budget=4 << 30))
    assert rep["failed"] == 0
    assert rep["state"]["max_in_flight"] >= 2          # batches overlapped on the device
    assert rep["p99_ms"] >= rep["p50_ms"] > 0
    for k, (w, pr) in enumerate(zip(ws, prods)):
        n = rep["done"][k]["n"]
        alone = P.polymul(pr["field_bits"], pr["f_exps"], pr["f_coefs"], pr["g_exps"], pr["g_coefs"])
        assert alone.n == n
        np.testing.assert_array_equal(alone.keys.cpu().numpy(), pr["out"][0][:n].cpu().numpy())
        np.testing.assert_array_equal(alone.coefs.cpu().numpy(), pr["out"][1][:n].cpu().numpy())
    rng = np.random.default_rng(1)
    sparse = [k for k, w in enumerate(ws) if w.f.n <= 8192]
    for k in rng.choice(sparse, size=15, replace=False):
        w = ws[k]
        e, c = oracle.mul(w.nvars, w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
        n = rep["done"][k]["n"]
        np.testing.assert_array_equal(prods[k]["out"][0][:n].cpu().numpy().view(np.uint64), pack_np(e, w.field_bits))
        np.testing.assert_array_equal(prods[k]["out"][1][:n].cpu().numpy().view(np.uint64), c)


def test_serving_budget_admission():
    """All requests queued at once under an HBM budget a third of what the
    whole stream needs as one batch: admission must split it into at least
    three batches, every request must succeed, and a request that cannot
    fit the budget alone must fail with PM_ENOMEM."""
    import paper_1303_7425_gb300 as P
    from paper_1303_7425_gb300.serving import serve
    ws, _ = _stream(count=40, dense=0, seed=23, rate=1e6, hi=400)
    prods = [_prod(w) for w in ws]
    whole = P.batch_workspace(prods)[0]
    alone = max(P.batch_workspace([p])[0] for p in prods)
    budget = max(alone, whole // 3)
    assert whole > 2 * budget                          # one batch cannot hold half the stream
    huge = polygen.sparse_product(polygen.Stream(99, 0), 4, 4096, 4096)     # 16.7M products
    ws.append(huge)
    prods.append(_prod(huge))
    assert P.batch_workspace([prods[-1]])[0] > budget
    t = [0.0] * len(ws)
    rep = serve(list(zip(t, prods)), [w.term_products for w in ws],
                server_kwargs=dict(streams=2, max_batch=64, device_budget=budget))
    assert rep["done"][len(ws) - 1]["status"] == -5
    assert all(rep["done"][k]["status"] == 0 for k in range(len(ws) - 1))
    assert rep["state"]["batches"] >= 3                # admission split the stream
    for k in range(0, len(ws) - 1, 7):
        w = ws[k]
        e, c = oracle.mul(w.nvars, w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
        n = rep["done"][k]["n"]
        np.testing.assert_array_equal(prods[k]["out"][1][:n].cpu().numpy().view(np.uint64), c)


def test_serving_cancellation():
    """Requests withdrawn before admission complete with PM_ECANCELED and
    leave their outputs untouched; the others complete exactly as computed
    alone; a tag that is unknown or already admitted cannot be cancelled."""
    import time

    import paper_1303_7425_gb300 as P
    ws, _ = _stream(count=30, dense=0, seed=31, rate=1e6, hi=300)
    prods = [_prod(w) for w in ws]
    srv = P.Server(device_budget=1 << 30, streams=2, max_batch=8)
    try:
        for k, pr in enumerate(prods):
            srv.submit(pr, k)
        cancel = set(range(1, 30, 3))
        for k in sorted(cancel):
            assert srv.cancel(k)
        assert not srv.cancel(1000)                  # unknown tag
        done = {}
        t0 = time.time()
        while len(done) < len(ws) and time.time() - t0 < 60:
            for d in srv.progress():
                done[d["tag"]] = d
        assert len(done) == len(ws)
        assert not srv.cancel(0)                     # finished: nothing to withdraw
    finally:
        srv.close()
    for k, pr in enumerate(prods):
        if k in cancel:
            assert done[k]["status"] == -9 and done[k]["n"] == 0
            assert bool((pr["out"][0] == -1).all()) and bool((pr["out"][1] == -1).all())
        else:
            assert done[k]["status"] == 0
            alone = P.polymul(pr["field_bits"], pr["f_exps"], pr["f_coefs"], pr["g_exps"], pr["g_coefs"])
            n = done[k]["n"]
            assert alone.n == n
            np.testing.assert_array_equal(alone.coefs.cpu().numpy(), pr["out"][1][:n].cpu().numpy())

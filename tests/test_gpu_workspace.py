"""The product on a caller-owned workspace (pm_workspace_size +
pm_polymul_ws): for every strategy and coefficient kind the result equals the
oracle bit for bit, the size query's bytes suffice, and a workspace that runs
out at any point of the call fails cleanly with PM_ENOMEM (the host-side form
of an allocation failure), after which the stream and the library still give
exact results."""

import numpy as np
import pytest

import oracle
import polygen
from tests.gpu_util import pack_np, to_dev

pytestmark = pytest.mark.gpu


def _cases():
    dense = polygen.monomials_total_degree(4, 8)
    st = polygen.Stream(41, 0)
    return {
        "sparse4v_auto": (polygen.workload_sparse4v(), {}),
        "dense4v_direct": (polygen.Workload("d", 4, [16] * 4, "m61", polygen.Poly(dense, st.coef_m61(len(dense))),
                                            polygen.Poly(dense[::-1].copy(), st.coef_m61(len(dense)))),
                           dict(strategy="direct")),
        "dense4v_i64_direct": (polygen.Workload("di", 4, [16] * 4, "i64",
                                                polygen.Poly(dense, st.coef_i64(len(dense), 1 << 40)),
                                                polygen.Poly(dense.copy(), st.coef_i64(len(dense), 1 << 40))),
                               dict(strategy="direct")),
        "sparse5_sort": (polygen.sparse_product(polygen.Stream(9, 0), 5, 1500, 900, 30), dict(strategy="sort")),
        "sparse3_hash": (polygen.sparse_product(polygen.Stream(12, 0), 3, 2000, 2000, 400), dict(strategy="hash")),
        "sparse5_bucket": (polygen.sparse_product(polygen.Stream(13, 0), 5, 1500, 900), dict(strategy="bucket")),
    }


def _out(cap, kind):
    import torch
    words = 1 if kind == "m61" else 2
    return (torch.full((cap,), -1, dtype=torch.int64, device="cuda"),
            torch.full((cap, words) if words == 2 else (cap,), -1, dtype=torch.int64, device="cuda"))


def _check(w, r):
    e, c = oracle.mul(w.nvars, w.field_bits, w.kind, w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
    assert r.n == len(e)
    np.testing.assert_array_equal(r.keys.cpu().numpy().view(np.uint64), pack_np(e, w.field_bits))
    np.testing.assert_array_equal(r.coefs.cpu().numpy().view(np.uint64).reshape(-1),
                                  np.asarray(c, dtype=np.uint64).reshape(-1))


@pytest.mark.parametrize("name", list(_cases()))
def test_workspace_product_equals_oracle(name):
    import torch

    import paper_1303_7425_gb300 as P
    w, opts = _cases()[name]
    f = to_dev(w.f.exps, w.f.coefs, w.kind)
    g = to_dev(w.g.exps, w.g.coefs, w.kind)
    nbytes, n = P.workspace_size(w.field_bits, f[0], f[1], g[0], g[1], kind=w.kind, **opts)
    assert nbytes > 0
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    out = _out(max(n, 1), w.kind)
    for _ in range(2):                         # the workspace keeps the first call's contents
        r = P.polymul_ws(w.field_bits, f[0], f[1], g[0], g[1], out, ws, kind=w.kind, **opts)
        torch.cuda.synchronize()
        assert r.n == n
        if opts.get("strategy"):
            assert r.stats["strategy"] == opts["strategy"]
        _check(w, r)


def test_workspace_exhausted_at_every_stage_fails_cleanly():
    """Workspaces cut short at many points of the call (before the operands,
    between the strategy's steps, just before the last block): each call
    returns PM_ENOMEM with h->n = 0 and nothing written past the workspace;
    a call with the full size on the same stream afterwards is exact."""
    import torch

    import paper_1303_7425_gb300 as P
    for name in ("sparse4v_auto", "dense4v_direct", "sparse3_hash", "sparse5_bucket"):
        w, opts = _cases()[name]
        f = to_dev(w.f.exps, w.f.coefs, w.kind)
        g = to_dev(w.g.exps, w.g.coefs, w.kind)
        nbytes, n = P.workspace_size(w.field_bits, f[0], f[1], g[0], g[1], kind=w.kind, **opts)
        guard = 1 << 16
        big = torch.full((nbytes + guard,), 0x5A, dtype=torch.uint8, device="cuda")
        out = _out(max(n, 1), w.kind)
        cuts = sorted({0, 256, nbytes // 8, nbytes // 3, nbytes // 2, (3 * nbytes) // 4,
                       max(0, nbytes - 4096), max(0, nbytes - 256)})
        # the hashed-window size carries a margin of one quarter: cut well below it
        cuts = [c - c % 256 for c in cuts if c < nbytes and not (name == "sparse3_hash" and c > nbytes // 2)]
        for cut in cuts:
            with pytest.raises(P.PolymulError) as ei:
                P.polymul_ws(w.field_bits, f[0], f[1], g[0], g[1], out, big[:cut], kind=w.kind, **opts)
            assert ei.value.code == -5, (name, cut, ei.value.code)
            torch.cuda.synchronize()
            # nothing past the workspace changed
            assert bool((big[cut:cut + guard] == 0x5A).all()), (name, cut)
            big[:].fill_(0x5A)
        r = P.polymul_ws(w.field_bits, f[0], f[1], g[0], g[1], out, big[:nbytes], kind=w.kind, **opts)
        torch.cuda.synchronize()
        _check(w, r)


def test_workspace_argument_errors():
    import torch

    import paper_1303_7425_gb300 as P
    w, _ = _cases()["sparse4v_auto"]
    f = to_dev(w.f.exps, w.f.coefs)
    g = to_dev(w.g.exps, w.g.coefs)
    nbytes, n = P.workspace_size(w.field_bits, f[0], f[1], g[0], g[1])
    ws = torch.empty(nbytes + 512, dtype=torch.uint8, device="cuda")
    out = _out(n, "m61")
    with pytest.raises(P.PolymulError) as ei:                       # not 256-byte aligned
        P.polymul_ws(w.field_bits, f[0], f[1], g[0], g[1], out, ws[8:8 + nbytes])
    assert ei.value.code == -1
    small = _out(max(n // 2, 1), "m61")
    with pytest.raises(P.PolymulError) as ei:                       # capacity, as for pm_polymul
        P.polymul_ws(w.field_bits, f[0], f[1], g[0], g[1], small, ws[:nbytes])
    assert ei.value.code == -4 and ei.value.needed == n
    empty = to_dev(np.zeros((0, 4), np.uint32), np.zeros(0, np.uint64))
    assert P.workspace_size(w.field_bits, empty[0], empty[1], g[0], g[1])[1] == 0

"""Slices of the output key space on one GPU (pm_shard_bounds +
pm_polymul_range, Alg. 2 of Sec. 3): the slices of consecutive shard bounds,
concatenated in order, equal the whole product and the oracle bit for bit,
for every strategy and both coefficient kinds; the shards' term-product
counts add up to n_f n_g and are balanced; arbitrary key slices (bounds that
are not monomials of the product's box) hold exactly the oracle's terms in
the slice.  The ranks run one after another here; across GPUs the slices are
gathered by paper_1303_7425_gb300.shard (tested on CPU ranks)."""

import numpy as np
import pytest

import oracle
import polygen
from tests.gpu_util import pack_np, to_dev

pytestmark = pytest.mark.gpu


def _cases():
    dense = polygen.monomials_total_degree(4, 10)
    st = polygen.Stream(77, 0)
    return {
        "sparse4v": (polygen.workload_sparse4v(), "auto"),
        "dense4v_direct": (polygen.Workload("d", 4, [16] * 4, "m61", polygen.Poly(dense, st.coef_m61(len(dense))),
                                            polygen.Poly(dense[::-1].copy(), st.coef_m61(len(dense)))), "direct"),
        "dense4v_i64": (polygen.Workload("di", 4, [16] * 4, "i64", polygen.Poly(dense, st.coef_i64(len(dense), 1 << 40)),
                                         polygen.Poly(dense.copy(), st.coef_i64(len(dense), 1 << 40))), "auto"),
        "sparse5_sort": (polygen.sparse_product(polygen.Stream(9, 0), 5, 1500, 900, 30), "sort"),
        "sparse3_hash": (polygen.sparse_product(polygen.Stream(12, 0), 3, 2000, 2000, 400), "hash"),
        "sparse5_bucket": (polygen.sparse_product(polygen.Stream(13, 0), 5, 1500, 900), "bucket"),
    }


def _np(r):
    c = r.coefs.cpu().numpy().view(np.uint64)
    return r.keys.cpu().numpy().view(np.uint64), (c.reshape(r.n, -1) if r.n else c.reshape(0, max(1, c.ndim)))


@pytest.mark.parametrize("name", list(_cases()))
@pytest.mark.parametrize("nshards", [2, 3, 5])
def test_shards_concatenate_to_the_product(name, nshards):
    import paper_1303_7425_gb300 as P
    w, strategy = _cases()[name]
    f = to_dev(w.f.exps, w.f.coefs, w.kind)
    g = to_dev(w.g.exps, w.g.coefs, w.kind)
    bounds, prods = P.shard_bounds(w.field_bits, f[0], f[1], g[0], g[1], nshards, kind=w.kind)
    assert bounds[0] == 0 and bounds[-1] == 2**64 - 1 and bounds == sorted(bounds)
    whole = P.polymul(w.field_bits, f[0], f[1], g[0], g[1], kind=w.kind, strategy=strategy)
    nf, ng = whole.stats["n_f"], whole.stats["n_g"]
    assert sum(prods) == nf * ng
    assert max(prods) <= 2 * nf * ng / nshards + nf * ng / 64
    keys, coefs = [], []
    for m in range(nshards):
        r = P.polymul_range(w.field_bits, f[0], f[1], g[0], g[1], bounds[m], bounds[m + 1], kind=w.kind,
                            strategy=strategy)
        k, c = _np(r)
        assert all(bounds[m] <= int(x) < bounds[m + 1] for x in k)
        keys.append(k)
        coefs.append(c)
    wk, wc = _np(whole)
    np.testing.assert_array_equal(np.concatenate(keys), wk)
    np.testing.assert_array_equal(np.concatenate(coefs), wc)
    e, c = oracle.mul(w.nvars, w.field_bits, w.kind, w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
    np.testing.assert_array_equal(wk, pack_np(e, w.field_bits))
    np.testing.assert_array_equal(wc.reshape(-1), np.asarray(c, dtype=np.uint64).reshape(-1))


@pytest.mark.parametrize("strategy", ["direct", "sort", "hash", "bucket"])
def test_arbitrary_key_slices(strategy):
    """Bounds drawn at random over the whole 64-bit range and near the
    product's keys, including keys whose fields lie outside the exponent box
    and keys with guard bits set."""
    import paper_1303_7425_gb300 as P
    w = polygen.sparse_product(polygen.Stream(21, 0), 3, 400, 300, 20)
    e, c = oracle.mul(w.nvars, w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
    keys = pack_np(e, w.field_bits)
    f = to_dev(w.f.exps, w.f.coefs)
    g = to_dev(w.g.exps, w.g.coefs)
    st = polygen.Stream(22, 0)
    picks = keys[st.below(keys.size, 12).astype(np.int64)]
    cands = sorted({0, 1, 2**64 - 1, int(keys[0]), int(keys[-1]), int(keys[-1]) + 1,
                    *(int(x) for x in picks), *(int(x) + 1 for x in picks), *(int(x) - 1 for x in picks),
                    *(int(x) for x in st.u64(6))})
    cands = [x for x in cands if 0 <= x < 2**64]
    rng = np.random.default_rng(5)
    for _ in range(16):
        i, j = sorted(int(x) for x in rng.choice(len(cands), 2, replace=False))   # indices: exact integers
        lo, hi = cands[i], cands[j]
        r = P.polymul_range(w.field_bits, f[0], f[1], g[0], g[1], lo, hi, strategy=strategy)
        sel = np.array([lo <= int(k) < hi for k in keys], dtype=bool)
        k, cc = _np(r)
        np.testing.assert_array_equal(k, keys[sel])
        np.testing.assert_array_equal(cc.reshape(-1), np.asarray(c, dtype=np.uint64)[sel])
    empty = P.polymul_range(w.field_bits, f[0], f[1], g[0], g[1], int(keys[-1]) + 1, 2**64 - 1, strategy=strategy)
    assert empty.n == 0


def test_sharded_polymul_one_rank_group_equals_the_product():
    """shard.sharded_polymul (the split, this rank's slice, the ordered
    gather) on a one-rank gloo group: the gathered result equals pm_polymul
    bit for bit, for both coefficient kinds."""
    import socket

    import torch.distributed as dist

    import paper_1303_7425_gb300 as P
    from paper_1303_7425_gb300.shard import sharded_polymul
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        for name in ("sparse4v", "dense4v_i64"):
            w, _ = _cases()[name]
            f = to_dev(w.f.exps, w.f.coefs, w.kind)
            g = to_dev(w.g.exps, w.g.coefs, w.kind)
            hk, hc, n, st = sharded_polymul(w.field_bits, f[0], f[1], g[0], g[1], kind=w.kind)
            whole = P.polymul(w.field_bits, f[0], f[1], g[0], g[1], kind=w.kind)
            assert n == whole.n and st["slice_terms"] == whole.n
            np.testing.assert_array_equal(hk.numpy(), whole.keys.cpu().numpy())
            np.testing.assert_array_equal(hc.numpy().reshape(-1), whole.coefs.cpu().numpy().reshape(-1))
    finally:
        dist.destroy_process_group()

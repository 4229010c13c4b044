"""The measured workloads at full size, compared with the oracle element by
element, in the launch configuration the benchmark times (a captured plan's
replay) and through the plain call:
  - the dense 4-variable product (112,911,876 term products, 135,751 terms),
    mod p and int64 -> int128, against the definition product (oracle_mul);
  - the sparse 5-variable product (2.5e9 term products), against the
    paper's Alg. 1 on all host threads (oracle_mul_alg1, itself pinned to the
    definition product in tests/test_oracle_pins.py)."""

import os

import numpy as np
import pytest

import oracle
import polygen
from tests.gpu_util import pack_np, to_dev

pytestmark = pytest.mark.gpu


def _same(keys, coefs, ref_e, ref_c, bits):
    assert keys.shape[0] == ref_e.shape[0]
    np.testing.assert_array_equal(keys, pack_np(ref_e, bits))
    np.testing.assert_array_equal(coefs.reshape(-1), np.asarray(ref_c, dtype=np.uint64).reshape(-1))


def _plan_and_plain(w):
    import torch

    import paper_1303_7425_gb300 as P
    f = to_dev(w.f.exps, w.f.coefs, w.kind)
    g = to_dev(w.g.exps, w.g.coefs, w.kind)
    cap = P.out_bound(w.field_bits, f[0], g[0])
    words = 1 if w.kind == "m61" else 2
    out = (torch.full((cap,), -1, dtype=torch.int64, device="cuda"),
           torch.full((cap, words) if words == 2 else (cap,), -1, dtype=torch.int64, device="cuda"))
    plan = P.Plan(w.field_bits, f[0], f[1], g[0], g[1], out, kind=w.kind)
    try:
        assert plan.captured
        out[0].fill_(-1)
        out[1].fill_(-1)
        plan.run()
        n = plan.finish()
        torch.cuda.synchronize()
        replay = (out[0][:n].cpu().numpy().view(np.uint64).copy(), out[1][:n].cpu().numpy().view(np.uint64).copy())
    finally:
        plan.close()
    r = P.polymul(w.field_bits, f[0], f[1], g[0], g[1], kind=w.kind)
    torch.cuda.synchronize()
    plain = (r.keys.cpu().numpy().view(np.uint64), r.coefs.cpu().numpy().view(np.uint64))
    return replay, plain


@pytest.mark.parametrize("kind", ["m61", "i64"])
def test_dense4v_full_size_every_term(kind):
    w = polygen.workload_dense4v(kind)
    replay, plain = _plan_and_plain(w)
    e, c = oracle.mul(w.nvars, w.field_bits, kind, w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
    assert e.shape[0] == 135751
    _same(*replay, e, c, w.field_bits)
    _same(*plain, e, c, w.field_bits)


def test_sparse5v_full_size_every_term():
    w = polygen.workload_sparse5v()
    replay, plain = _plan_and_plain(w)
    e, c, _ = oracle.mul_alg1(w.nvars, w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs, l=64,
                              threads=os.cpu_count() or 1)
    assert e.shape[0] == 3824065
    _same(*replay, e, c, w.field_bits)
    _same(*plain, e, c, w.field_bits)

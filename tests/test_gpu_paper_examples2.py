"""The paper's Examples 2 and 3 at full size (Sec. 6), through the hashed
windows: 2.0e10 and 5.6e10 term products, results of 312,855,140 and
144,049,555 terms.  Pinned by the term counts the paper prints
(tests/golden/paper_counts.txt), by the oracle's coefficient at sampled
result monomials, and over the whole result by evaluation at points whose
coordinates are powers of two, h(r) = f(r) g(r) mod p (eval_pow2: no
library or oracle code involved)."""

import numpy as np
import pytest

import oracle
import polygen
from tests.gpu_util import P61, check_canonical, eval_pow2, unpack_np

pytestmark = pytest.mark.gpu


def _golden_count(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")
    for line in open(path):
        parts = line.split()
        if parts and parts[0] == name:
            return int(parts[3])
    raise KeyError(name)


@pytest.mark.parametrize("name", ["ex2", "ex3"])
def test_paper_examples_2_and_3_full_size(name):
    import torch
    import paper_1303_7425_gb300 as P
    from tests.gpu_util import to_dev
    w = polygen.paper_example(name)
    f = to_dev(w.f.exps, w.f.coefs)
    g = to_dev(w.g.exps, w.g.coefs)
    n_expect = _golden_count(name)
    out = (torch.empty(n_expect + 16, dtype=torch.int64, device="cuda"),
           torch.empty(n_expect + 16, dtype=torch.int64, device="cuda"))
    r = P.polymul(w.field_bits, f[0], f[1], g[0], g[1], out=out)
    torch.cuda.synchronize()
    assert r.stats["strategy"] == "hash"
    assert r.n == n_expect
    rng = np.random.default_rng(7)
    # keys ascending and canonical on a few million-term stretches
    for start in rng.integers(0, r.n - 2_000_000, size=3):
        keys = r.keys[start:start + 2_000_000].cpu().numpy().view(np.uint64)
        coefs = r.coefs[start:start + 2_000_000].cpu().numpy().view(np.uint64)
        check_canonical(keys, coefs, w.field_bits)
    # sampled coefficients against the oracle
    idx = np.sort(rng.choice(r.n, size=300, replace=False))
    it = torch.from_numpy(idx).cuda()
    skeys = r.keys[it].cpu().numpy().view(np.uint64)
    scoefs = r.coefs[it].cpu().numpy().view(np.uint64)
    want = oracle.coef_at(w.nvars, w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs,
                          unpack_np(skeys, w.field_bits))
    np.testing.assert_array_equal(scoefs, np.asarray(want, dtype=np.uint64))
    # the whole result at points (2^a_1, ..., 2^a_5), in chunks
    for _ in range(3):
        a = [int(x) for x in rng.integers(1, 61, size=w.nvars)]
        hv = 0
        for s0 in range(0, r.n, 20_000_000):
            ck = r.keys[s0:s0 + 20_000_000].cpu().numpy().view(np.uint64)
            cc = r.coefs[s0:s0 + 20_000_000].cpu().numpy().view(np.uint64)
            hv = (hv + eval_pow2(unpack_np(ck, w.field_bits), cc, a)) % P61
        fv = eval_pow2(w.f.exps, w.f.coefs, a)
        gv = eval_pow2(w.g.exps, w.g.coefs, a)
        assert hv == fv * gv % P61

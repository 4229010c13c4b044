"""The paper's Example 1 at full size (Sec. 6): f1 = (1+x+y+z+t)^40 times
g1 = f1 + 1, 1.84e10 term products.  Pinned by the term count the paper
prints (1,929,501 = C(84, 4), tests/golden/paper_counts.txt) and, for every
result term, by the closed form h = f1^2 + f1 = (1+x+y+z+t)^80 +
(1+x+y+z+t)^40: the coefficient of x^a y^b z^c t^d is the multinomial
80! / (a! b! c! d! (80-s)!) plus, when s = a+b+c+d <= 40, the one of
degree 40, all mod 2^61 - 1 -- no oracle run needed."""

import numpy as np
import pytest

import polygen
from tests.gpu_util import P61, check_canonical, unpack_np

pytestmark = pytest.mark.gpu


def _golden_count(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")
    for line in open(path):
        parts = line.split()
        if parts and parts[0] == name:
            return int(parts[3])
    raise KeyError(name)


def _closed_form(exps):
    fact = [1] * 81
    for k in range(1, 81):
        fact[k] = fact[k - 1] * k % P61
    inv = [pow(f, P61 - 2, P61) for f in fact]
    out = np.empty(len(exps), dtype=np.uint64)
    for q, (a, b, c, d) in enumerate(exps.tolist()):
        s = a + b + c + d
        v = fact[80] * inv[a] % P61 * inv[b] % P61 * inv[c] % P61 * inv[d] % P61 * inv[80 - s] % P61
        if s <= 40:
            v = (v + fact[40] * inv[a] % P61 * inv[b] % P61 * inv[c] % P61 * inv[d] % P61 * inv[40 - s]) % P61
        out[q] = v
    return out


def test_paper_example1_full_size():
    import torch
    import paper_1303_7425_gb300 as P
    from tests.gpu_util import to_dev
    w = polygen.paper_example1()
    assert w.f.n == 135751 and w.g.n == 135751
    f = to_dev(w.f.exps, w.f.coefs)
    g = to_dev(w.g.exps, w.g.coefs)
    r = P.polymul(w.field_bits, f[0], f[1], g[0], g[1])
    torch.cuda.synchronize()
    assert r.stats["strategy"] == "direct"
    assert r.n == _golden_count("ex1")
    keys = r.keys.cpu().numpy().view(np.uint64)
    coefs = r.coefs.cpu().numpy().view(np.uint64)
    check_canonical(keys, coefs, w.field_bits)
    exps = unpack_np(keys, w.field_bits)
    assert int(exps.sum(axis=1).max()) == 80
    np.testing.assert_array_equal(coefs, _closed_form(exps))

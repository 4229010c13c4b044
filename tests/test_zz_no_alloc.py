"""pm_polymul_noalloc, the entry point for callers that cannot allocate
device memory (its scratch is a static device array inside the library).
Its results must equal pm_polymul's bit for bit, on two calls in a row: the
second call also shows that the scratch left over by the first does not leak
into the next result.  This file is collected last on purpose."""

import numpy as np
import pytest

import oracle
import polygen
from tests.gpu_util import pack_np, to_dev

pytestmark = pytest.mark.gpu


def _inputs(seed, nv, nf, ng, kind):
    st = polygen.Stream(seed, 0)
    fe = st.below(6, nf * nv).astype(np.uint32).reshape(nf, nv)       # repeats and a dense support
    ge = st.below(6, ng * nv).astype(np.uint32).reshape(ng, nv)
    if kind == "m61":
        fc, gc = st.coef_m61(nf), st.coef_m61(ng)
    else:
        fc, gc = st.coef_i64(nf, 1 << 40), st.coef_i64(ng, 1 << 40)
    return fe, fc, ge, gc


def _run_both(bits, kind, fe, fc, ge, gc):
    import torch

    import paper_1303_7425_gb300 as P
    f = to_dev(fe, fc, kind)
    g = to_dev(ge, gc, kind)
    ref = P.polymul(bits, f[0], f[1], g[0], g[1], kind=kind)
    cap = fe.shape[0] * ge.shape[0]
    words = 1 if kind == "m61" else 2
    out = (torch.full((cap,), -1, dtype=torch.int64, device="cuda"),
           torch.full((cap, words) if words == 2 else (cap,), -1, dtype=torch.int64, device="cuda"))
    n = P.polymul_noalloc(bits, f[0], f[1], g[0], g[1], out, kind=kind)
    torch.cuda.synchronize()
    assert n == ref.n
    np.testing.assert_array_equal(out[0][:n].cpu().numpy(), ref.keys.cpu().numpy())
    np.testing.assert_array_equal(out[1][:n].cpu().numpy(), ref.coefs.cpu().numpy())
    return out, n


@pytest.mark.parametrize("kind", ["m61", "i64"])
def test_noalloc_matches_polymul_twice(kind):
    bits = [10, 10, 10]
    a = _inputs(7, 3, 200, 300, kind)
    b = _inputs(8, 3, 64, 900, kind)      # a different shape on the second call
    out1, n1 = _run_both(bits, kind, *a)
    out2, n2 = _run_both(bits, kind, *b)
    # and against the oracle, once
    e, c = oracle.mul(3, bits, kind, *b)
    np.testing.assert_array_equal(out2[0][:n2].cpu().numpy().view(np.uint64), pack_np(e, bits))
    np.testing.assert_array_equal(out2[1][:n2].cpu().numpy().view(np.uint64).reshape(-1),
                                  np.asarray(c, dtype=np.uint64).reshape(-1))


def test_noalloc_limits_and_errors():
    import torch

    import paper_1303_7425_gb300 as P
    bits = [8, 8]
    st = polygen.Stream(9, 0)
    big = st.below(50, 2 * 4097).astype(np.uint32).reshape(4097, 2)
    f = to_dev(big, st.coef_m61(4097))
    g = to_dev(big[:3], st.coef_m61(3))
    out = (torch.empty(16, dtype=torch.int64, device="cuda"), torch.empty(16, dtype=torch.int64, device="cuda"))
    with pytest.raises(P.PolymulError) as ei:                 # more terms than the static scratch holds
        P.polymul_noalloc(bits, f[0], f[1], g[0], g[1], out)
    assert ei.value.code == -1
    f = to_dev(big[:300], st.coef_m61(300))
    g = to_dev(big[:300], st.coef_m61(300))
    with pytest.raises(P.PolymulError) as ei:                 # 90,000 products > 65,536
        P.polymul_noalloc(bits, f[0], f[1], g[0], g[1], out)
    assert ei.value.code == -1
    g = to_dev(big[:200], st.coef_m61(200))
    with pytest.raises(P.PolymulError) as ei:                 # output capacity reported like pm_polymul
        P.polymul_noalloc(bits, f[0], f[1], g[0], g[1], out)
    assert ei.value.code == -4 and ei.value.needed > 16
    one = np.array([1], np.uint64)
    f = to_dev(np.array([[100, 0]], np.uint32), one)
    g = to_dev(np.array([[100, 0]], np.uint32), one)
    with pytest.raises(P.PolymulError) as ei:                 # the exponent guard rule
        P.polymul_noalloc(bits, f[0], f[1], g[0], g[1], out)
    assert ei.value.code == -2

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


def _codes_both(bits, kind, fe, fc, ge, gc):
    """(pm_polymul's code, its n) and (pm_polymul_noalloc's code, its n) on
    the same inputs; 0 and the result size when a call succeeds."""
    import torch

    import paper_1303_7425_gb300 as P
    f = to_dev(fe, fc, kind)
    g = to_dev(ge, gc, kind)
    words = 1 if kind == "m61" else 2
    cap = max(fe.shape[0] * ge.shape[0], 1)
    res = []
    for call in ("polymul", "noalloc"):
        out = (torch.full((cap,), -1, dtype=torch.int64, device="cuda"),
               torch.full((cap, words) if words == 2 else (cap,), -1, dtype=torch.int64, device="cuda"))
        try:
            if call == "polymul":
                n = P.polymul(bits, f[0], f[1], g[0], g[1], kind=kind, out=out).n
            else:
                n = P.polymul_noalloc(bits, f[0], f[1], g[0], g[1], out, kind=kind)
            res.append((0, n, out))
        except P.PolymulError as e:
            res.append((e.code, None, out))
    torch.cuda.synchronize()
    return res


def test_noalloc_int64_coefficient_bound_matches_polymul():
    """Both int64 refusals of the no-allocation kernel (a repeated input
    monomial whose sum leaves int64; max|a| max|b| min(n_f, n_g) above
    2^127 - 1) give pm_polymul's code."""
    bits = [8, 8]
    two = np.array([[3, 1], [3, 1]], np.uint32)                         # one monomial, twice
    other = np.array([[0, 0], [1, 0]], np.uint32)
    cases = [
        (two, np.array([2**62, 2**62], np.int64), other, np.array([5, 7], np.int64)),       # 2^63 leaves int64
        (other, np.array([5, 7], np.int64), two, np.array([-2**63, -1], np.int64)),          # in g, below
        (other, np.array([-2**63, 3], np.int64), other, np.array([-2**63, 1], np.int64)),    # 2^126 * 2 > bound
        (three := np.array([[0, 0], [1, 0], [2, 0]], np.uint32), np.array([2**63 - 1, 1, 1], np.int64), three,
         np.array([-2**63 + 1, 1, 1], np.int64)),                                               # ~2^126 * 3
    ]
    for fe, fc, ge, gc in cases:
        (c0, _, _), (c1, _, _) = _codes_both(bits, "i64", fe, fc, ge, gc)
        assert c0 == -3 and c1 == -3, (c0, c1)
    # just inside the bound: (2^63 - 1)^2 * 1 < 2^127 - 1 with one-term operands
    fe = np.array([[1, 2]], np.uint32)
    (c0, n0, o0), (c1, n1, o1) = _codes_both(bits, "i64", fe, np.array([2**63 - 1], np.int64), fe,
                                             np.array([-(2**63 - 1)], np.int64))
    assert c0 == 0 and c1 == 0 and n0 == n1 == 1
    assert np.array_equal(o0[1][:1].cpu().numpy(), o1[1][:1].cpu().numpy())


@pytest.mark.parametrize("kind", ["m61", "i64"])
def test_noalloc_cancelling_operands(kind):
    """Repeated terms that cancel: an operand that cancels completely gives
    an empty result (PM_OK, n = 0); one that cancels in part gives
    pm_polymul's result."""
    bits = [10, 10, 10]
    P61 = (1 << 61) - 1
    fe = np.array([[1, 2, 3], [1, 2, 3], [0, 0, 1], [0, 0, 1]], np.uint32)
    if kind == "m61":
        fc = np.array([5, P61 - 5, 9, 2 * P61 - 9], np.uint64)          # each pair sums to 0 mod p
    else:
        fc = np.array([5, -5, 9, -9], np.int64)
    ge = np.array([[2, 0, 0], [0, 4, 0]], np.uint32)
    gc = np.array([3, 4], np.uint64 if kind == "m61" else np.int64)
    (c0, n0, _), (c1, n1, _) = _codes_both(bits, kind, fe, fc, ge, gc)
    assert (c0, n0) == (0, 0) and (c1, n1) == (0, 0)
    fe2 = np.concatenate([fe, np.array([[7, 7, 7]], np.uint32)])
    fc2 = np.concatenate([fc, np.array([11], fc.dtype)])
    (c0, n0, o0), (c1, n1, o1) = _codes_both(bits, kind, fe2, fc2, ge, gc)
    assert c0 == 0 and c1 == 0 and n0 == n1 == 2
    np.testing.assert_array_equal(o0[0][:2].cpu().numpy(), o1[0][:2].cpu().numpy())
    np.testing.assert_array_equal(o0[1][:2].cpu().numpy(), o1[1][:2].cpu().numpy())


def test_noalloc_error_order_matches_polymul():
    """Where two error rules apply at once, both entry points report the same
    one."""
    bits = [4, 4]
    dup = np.array([[1, 0], [1, 0]], np.uint32)
    big = np.array([[7, 0]], np.uint32)                                   # 1 + 7 reaches the guard bit 8
    over = np.array([[8, 0]], np.uint32)                                  # an input at the guard bit
    cases = [
        (dup, np.array([2**62, 2**62], np.int64), big, np.array([1], np.int64)),     # sum overflow + product exp
        (dup, np.array([2**62, 2**62], np.int64), over, np.array([1], np.int64)),    # sum overflow + input exp
        (np.array([[7, 0], [0, 1]], np.uint32), np.array([-2**63, -2**63], np.int64),
         np.array([[1, 0], [2, 0]], np.uint32), np.array([-2**63, -2**63], np.int64)),  # product exp + int128 bound
    ]
    expected = [-3, -2, -2]
    for (fe, fc, ge, gc), want in zip(cases, expected):
        (c0, _, _), (c1, _, _) = _codes_both(bits, "i64", fe, fc, ge, gc)
        assert c0 == want and c1 == want, (c0, c1, want)

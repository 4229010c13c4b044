"""Test-side helpers for the GPU parity tests: moving seeded workloads to the
device, decoding results, and packing oracle exponent vectors for
comparison.  Independent of both the oracle's arithmetic and the library."""

import numpy as np

P61 = (1 << 61) - 1


def pack_np(exps, bits):
    """Pack (n, nvars) exponent rows the way include/polymul.h documents
    (x_1 in the most significant field)."""
    exps = np.asarray(exps, dtype=np.uint64)
    nv = len(bits)
    off = [sum(bits[v + 1:]) for v in range(nv)]
    k = np.zeros(exps.shape[0], dtype=np.uint64)
    for v in range(nv):
        k |= exps[:, v] << np.uint64(off[v])
    return k


def unpack_np(keys, bits):
    keys = np.asarray(keys, dtype=np.uint64)
    nv = len(bits)
    off = [sum(bits[v + 1:]) for v in range(nv)]
    out = np.zeros((keys.shape[0], nv), dtype=np.uint32)
    for v in range(nv):
        out[:, v] = (keys >> np.uint64(off[v])) & np.uint64((1 << bits[v]) - 1)
    return out


def to_dev(exps, coefs, kind="m61"):
    import torch
    e = torch.from_numpy(np.ascontiguousarray(exps, dtype=np.uint32).view(np.int32)).cuda()
    if kind == "m61":
        c = torch.from_numpy(np.ascontiguousarray(coefs, dtype=np.uint64).view(np.int64)).cuda()
    else:
        c = torch.from_numpy(np.ascontiguousarray(coefs, dtype=np.int64)).cuda()
    return e, c


def run_gpu(bits, kind, fe, fc, ge, gc, **kw):
    """Product through the C-ABI; returns (keys uint64, coefs uint64 or (n,2)
    uint64, stats)."""
    import paper_1303_7425_gb300 as P
    import torch
    f = to_dev(fe, fc, kind)
    g = to_dev(ge, gc, kind)
    r = P.polymul(bits, f[0], f[1], g[0], g[1], kind=kind, **kw)
    torch.cuda.synchronize()
    keys = r.keys.cpu().numpy().view(np.uint64)
    coefs = r.coefs.cpu().numpy().view(np.uint64)
    return keys, coefs, r.stats


def assert_same(gpu, ref, bits):
    keys, coefs, _ = gpu
    rexps, rcoefs = ref
    rkeys = pack_np(rexps, bits)
    assert keys.shape == rkeys.shape, (keys.shape, rkeys.shape)
    np.testing.assert_array_equal(keys, rkeys)
    np.testing.assert_array_equal(coefs.reshape(-1), np.asarray(rcoefs, dtype=np.uint64).reshape(-1))


def check_canonical(keys, coefs, bits, kind="m61"):
    """Properties of any correct result: strictly ascending keys, no zero
    coefficient, residues below p, guard bits clear."""
    if keys.size > 1:
        assert np.all(keys[1:] > keys[:-1])
    if kind == "m61":
        assert np.all(coefs != 0) and np.all(coefs < np.uint64(P61))
    else:
        c = coefs.reshape(-1, 2)
        assert np.all((c[:, 0] | c[:, 1]) != 0)
    guard = np.uint64(0)
    off = 0
    for w in reversed(bits):
        guard |= np.uint64(1 << (off + w - 1))
        off += w
    assert not np.any(keys & guard)


def eval_pow2(exps, coefs, a):
    """p(2^a_1, ..., 2^a_n) mod 2^61 - 1 for a polynomial with residue
    coefficients: since 2^61 = 1 (mod 2^61 - 1), each term's value is its
    coefficient rotated left by (a . e) mod 61 bits inside 61 bits."""
    e = np.asarray(exps, dtype=np.uint64)
    k = (e @ np.asarray(a, dtype=np.uint64)) % np.uint64(61)
    c = np.asarray(coefs, dtype=np.uint64)
    rot = ((c << k) & np.uint64(P61)) | (c >> (np.uint64(61) - k))
    lo = int((rot & np.uint64((1 << 31) - 1)).sum(dtype=np.uint64))
    hi = int((rot >> np.uint64(31)).sum(dtype=np.uint64))
    return (lo + (hi << 31)) % P61

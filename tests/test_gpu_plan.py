"""Plans (pm_plan_*): the whole device path of one product captured into a
CUDA graph and replayed.  Every replay must equal the oracle on the current
inputs (bit-exact); inputs whose statistics leave the recorded ones must be
reported (PM_EPLAN) without touching memory out of bounds; a replay whose
result outgrows the capacity must be reported (PM_ECAPACITY)."""

import numpy as np
import pytest

import oracle
import polygen
from tests.gpu_util import pack_np, to_dev

pytestmark = pytest.mark.gpu

P61 = (1 << 61) - 1


def _dense(nvars=4, deg=8, seed=3, kind="m61"):
    mons = polygen.monomials_total_degree(nvars, deg)
    st = polygen.Stream(seed, 0)
    if kind == "m61":
        fc, gc = st.coef_m61(len(mons)), st.coef_m61(len(mons))
    else:
        fc, gc = st.coef_i64(len(mons), 1 << 20), st.coef_i64(len(mons), 1 << 20)
    return polygen.Workload(f"dense{nvars}v{deg}", nvars, [16] * nvars, kind, polygen.Poly(mons, fc),
                            polygen.Poly(mons[::-1].copy(), gc))


def _make(w, cap=None):
    import torch
    f = to_dev(w.f.exps, w.f.coefs, w.kind)
    g = to_dev(w.g.exps, w.g.coefs, w.kind)
    cap = cap if cap is not None else max(w.f.n * w.g.n, 1)
    words = 1 if w.kind == "m61" else 2
    out = (torch.full((cap,), -1, dtype=torch.int64, device="cuda"),
           torch.full((cap, 2) if words == 2 else (cap,), -1, dtype=torch.int64, device="cuda"))
    return f, g, out


def _expect(w, n, out):
    e, c = oracle.mul(w.nvars, w.field_bits, w.kind, w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
    assert n == len(e)
    np.testing.assert_array_equal(out[0][:n].cpu().numpy().view(np.uint64), pack_np(e, w.field_bits))
    np.testing.assert_array_equal(out[1][:n].cpu().numpy().view(np.uint64).reshape(-1),
                                  np.asarray(c, dtype=np.uint64).reshape(-1))


@pytest.mark.parametrize("kind", ["m61", "i64"])
def test_plan_replays_equal_oracle(kind):
    import paper_1303_7425_gb300 as P
    w = _dense(kind=kind)
    f, g, out = _make(w)
    plan = P.Plan(w.field_bits, f[0], f[1], g[0], g[1], out, kind=kind)
    try:
        assert plan.captured
        _expect(w, plan.n, out)
        out[0].fill_(-1)
        out[1].fill_(-1)
        for _ in range(3):
            plan.run()
        n = plan.finish()
        _expect(w, n, out)
    finally:
        plan.close()


def test_plan_dense_workload_equals_plain_call():
    """The 10,626 x 10,626 dense product: replays equal pm_polymul."""
    import paper_1303_7425_gb300 as P
    w = polygen.workload_dense4v()
    f, g, out = _make(w, cap=200_000)
    plan = P.Plan(w.field_bits, f[0], f[1], g[0], g[1], out)
    try:
        assert plan.captured and plan.n == 135751
        out[1].fill_(0)
        plan.run()
        n = plan.finish()
        ref = P.polymul(w.field_bits, f[0], f[1], g[0], g[1])
        assert n == ref.n
        assert bool((out[0][:n] == ref.keys).all()) and bool((out[1][:n] == ref.coefs).all())
    finally:
        plan.close()


def test_plan_recomputes_after_coefficient_change():
    import paper_1303_7425_gb300 as P
    w = _dense(seed=11)
    f, g, out = _make(w)
    plan = P.Plan(w.field_bits, f[0], f[1], g[0], g[1], out)
    try:
        for seed in (21, 22):
            w.f.coefs = polygen.Stream(seed, 1).coef_m61(w.f.n)
            w.g.coefs = polygen.Stream(seed, 2).coef_m61(w.g.n)
            f[1].copy_(to_dev(w.f.exps, w.f.coefs)[1])
            g[1].copy_(to_dev(w.g.exps, w.g.coefs)[1])
            plan.run()
            _expect(w, plan.finish(), out)
    finally:
        plan.close()


def test_plan_same_statistics_new_order():
    """Permuting the input terms keeps maxima, sizes and extreme monomials,
    so the replay stays exact."""
    import paper_1303_7425_gb300 as P
    w = _dense(seed=5)
    f, g, out = _make(w)
    plan = P.Plan(w.field_bits, f[0], f[1], g[0], g[1], out)
    try:
        perm = np.random.default_rng(0).permutation(w.f.n)
        w.f.exps = np.ascontiguousarray(w.f.exps[perm])
        w.f.coefs = np.ascontiguousarray(w.f.coefs[perm])
        fe, fc = to_dev(w.f.exps, w.f.coefs)
        f[0].copy_(fe)
        f[1].copy_(fc)
        plan.run()
        _expect(w, plan.finish(), out)
    finally:
        plan.close()


def test_plan_reports_changed_shape_then_recovers():
    import paper_1303_7425_gb300 as P
    w = _dense(seed=7)
    f, g, out = _make(w)
    plan = P.Plan(w.field_bits, f[0], f[1], g[0], g[1], out)
    try:
        saved = f[0].clone()
        # raise one exponent past the recorded maximum (still below the guard)
        bumped = w.f.exps.copy()
        bumped[0, 0] = 100
        f[0].copy_(to_dev(bumped, w.f.coefs)[0])
        plan.run()
        with pytest.raises(P.PolymulError) as ei:
            plan.finish()
        assert ei.value.code == -8
        # a term whose coefficient cancels to zero changes the canonical size
        f[0].copy_(saved)
        zc = w.f.coefs.copy()
        zc[len(zc) // 2] = 0
        f[1].copy_(to_dev(w.f.exps, zc)[1])
        plan.run()
        with pytest.raises(P.PolymulError) as ei:
            plan.finish()
        assert ei.value.code == -8
        # the recorded inputs again: exact
        f[1].copy_(to_dev(w.f.exps, w.f.coefs)[1])
        plan.run()
        _expect(w, plan.finish(), out)
    finally:
        plan.close()


def test_plan_capacity_reported():
    """f = x + 1, g = x - 1 gives x^2 - 1 (two terms, the capacity); with
    g = x + 1 the replay's result has three terms and must not be written."""
    import paper_1303_7425_gb300 as P
    e = np.array([[1], [0]], np.uint32)
    one = np.array([1, 1], np.uint64)
    w = polygen.Workload("cap", 1, [8], "m61", polygen.Poly(e, one),
                         polygen.Poly(e.copy(), np.array([1, P61 - 1], np.uint64)))
    f, g, out = _make(w, cap=2)
    plan = P.Plan(w.field_bits, f[0], f[1], g[0], g[1], out)
    try:
        assert plan.n == 2 and plan.captured
        g[1].copy_(to_dev(e, one)[1])
        out[0].fill_(-7)
        plan.run()
        with pytest.raises(P.PolymulError) as ei:
            plan.finish()
        assert ei.value.code == -4 and ei.value.needed == 3
        assert bool((out[0] == -7).all())          # nothing written
    finally:
        plan.close()


def test_plan_sort_strategy_runs_plain_calls():
    import paper_1303_7425_gb300 as P
    w = polygen.sparse_product(polygen.Stream(41, 0), 5, 300, 200)
    f, g, out = _make(w)
    plan = P.Plan(w.field_bits, f[0], f[1], g[0], g[1], out)
    try:
        assert not plan.captured
        _expect(w, plan.n, out)
        plan.run()
        _expect(w, plan.finish(), out)
    finally:
        plan.close()


@pytest.mark.parametrize("kind", ["m61", "i64"])
def test_plan_finish_to_host_equals_device_result(kind):
    """The replay's result copied on the device side into page-locked host
    buffers equals the device result; the host waits once."""
    import torch
    import paper_1303_7425_gb300 as P
    w = _dense(kind=kind, seed=13)
    f, g, out = _make(w)
    plan = P.Plan(w.field_bits, f[0], f[1], g[0], g[1], out, kind=kind)
    try:
        cap = out[0].shape[0]
        hk = torch.full((cap,), -1, dtype=torch.int64).pin_memory()
        hc = torch.full(tuple(out[1].shape), -1, dtype=torch.int64).pin_memory()
        for _ in range(2):
            plan.run()
            n = plan.finish_to_host(hk, hc)
            _expect(w, n, out)
            assert torch.equal(hk[:n], out[0][:n].cpu()) and torch.equal(hc[:n], out[1][:n].cpu())
        # a host buffer smaller than the result: nothing copied, size reported
        small_k = torch.full((n - 1,), -5, dtype=torch.int64).pin_memory()
        small_c = torch.full((n - 1,) + tuple(out[1].shape[1:]), -5, dtype=torch.int64).pin_memory()
        plan.run()
        with pytest.raises(P.PolymulError) as ei:
            plan.finish_to_host(small_k, small_c)
        assert ei.value.code == -4 and ei.value.needed == n
        assert bool((small_k == -5).all())
        # pageable host memory is refused
        with pytest.raises(P.PolymulError) as ei:
            plan.finish_to_host(torch.empty(cap, dtype=torch.int64), hc)
        assert ei.value.code == -1
    finally:
        plan.close()


def test_plan_finish_to_host_sort_strategy_plain_calls():
    import torch
    import paper_1303_7425_gb300 as P
    w = polygen.sparse_product(polygen.Stream(43, 0), 5, 200, 150)
    f, g, out = _make(w)
    plan = P.Plan(w.field_bits, f[0], f[1], g[0], g[1], out)
    try:
        assert not plan.captured
        hk = torch.empty(out[0].shape[0], dtype=torch.int64).pin_memory()
        hc = torch.empty(out[1].shape[0], dtype=torch.int64).pin_memory()
        plan.run()
        n = plan.finish_to_host(hk, hc)
        _expect(w, n, out)
        assert torch.equal(hk[:n], out[0][:n].cpu()) and torch.equal(hc[:n], out[1][:n].cpu())
    finally:
        plan.close()

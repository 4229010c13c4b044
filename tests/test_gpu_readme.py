"""The README's quick start, run as written: (3 + x y^2)(5 x + y) =
15 x + 3 y + 5 x^2 y^2 + x y^3, through polymul, unpack and a plan."""

import pytest

pytestmark = pytest.mark.gpu


def test_readme_quick_start():
    import torch
    import paper_1303_7425_gb300 as P
    bits = [16, 16]
    fe = torch.tensor([[0, 0], [1, 2]], dtype=torch.int32, device="cuda")
    fc = torch.tensor([3, 1], dtype=torch.int64, device="cuda")
    ge = torch.tensor([[1, 0], [0, 1]], dtype=torch.int32, device="cuda")
    gc = torch.tensor([5, 1], dtype=torch.int64, device="cuda")
    h = P.polymul(bits, fe, fc, ge, gc)
    exps = P.unpack(bits, h.keys)
    got = {tuple(e): int(c) for e, c in zip(exps.cpu().tolist(), h.coefs.cpu().tolist())}
    # ascending in lex order with x first: y < x < x y^3 < x^2 y^2
    assert [tuple(e) for e in exps.cpu().tolist()] == [(0, 1), (1, 0), (1, 3), (2, 2)]
    assert got == {(0, 1): 3, (1, 0): 15, (1, 3): 1, (2, 2): 5}
    cap = P.out_bound(bits, fe, ge)
    out = (torch.empty(cap, dtype=torch.int64, device="cuda"), torch.empty(cap, dtype=torch.int64, device="cuda"))
    plan = P.Plan(bits, fe, fc, ge, gc, out)
    try:
        plan.run()
        n = plan.finish()
        assert n == 4
        assert torch.equal(out[0][:n], h.keys) and torch.equal(out[1][:n], h.coefs)
    finally:
        plan.close()

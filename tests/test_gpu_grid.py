"""Step 1 of Alg. 1 on the GPU (pm_grid, the k_grid kernel): the splitters of
the Sec. 5 almost regular grid plus gamma_end, sorted and deduplicated, equal
the oracle's grid (oracle_grid, pinned by the hand-derived fixture
tests/golden/grid_sec5_16x16_l4.txt) bit for bit.  The direct strategy's
cost histogram (k_grid_hist) and the batched plan kernel (kb_plan) enumerate
their sample points with the same device function, grid_point."""

import os

import numpy as np
import pytest

import oracle
import polygen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _keys(st, n, hi=1 << 40):
    k = np.unique(st.below(hi, 3 * n + 8))
    return np.sort(k[st.permutation(k.size)[:n]]).astype(np.uint64)


def _expect(a, b, l):
    pts = oracle.grid(a, b, l)
    end = np.uint64(int(a[-1]) + int(b[-1]) + 1)
    return np.unique(np.concatenate([pts, np.array([end], np.uint64)]))


def _gpu(a, b, l):
    import torch

    import paper_1303_7425_gb300 as P
    da = torch.from_numpy(a.view(np.int64)).cuda()
    db = torch.from_numpy(b.view(np.int64)).cuda()
    return P.grid(da, db, l).cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("na,nb", [(1000, 777), (16, 16), (3, 500), (1, 1), (4096, 37), (65, 64)])
@pytest.mark.parametrize("l", [1, 4, 64, 200])
def test_grid_equals_oracle(na, nb, l):
    st = polygen.Stream(na * 7919 + nb * 31 + l, 0)
    a, b = _keys(st, na), _keys(st, nb)
    np.testing.assert_array_equal(_gpu(a, b, l), _expect(a, b, l))


def test_grid_on_the_hand_derived_fixture():
    """The 16 x 16, l = 4 grid written out by hand from Sec. 5 (1-based
    (i, j) pairs): keys chosen so every point alpha_i + beta_j is distinct
    and decodes back to (i, j)."""
    want = []
    with open(os.path.join(GOLDEN, "grid_sec5_16x16_l4.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                i, j = line.split()
                want.append(int(i) * 1000 + int(j))
    a = np.arange(1, 17, dtype=np.uint64) * np.uint64(1000)
    b = np.arange(1, 17, dtype=np.uint64)
    got = _gpu(a, b, 4)
    assert int(got[-1]) == 16 * 1000 + 16 + 1                   # gamma_end
    np.testing.assert_array_equal(got[:-1], np.unique(np.array(want, np.uint64)))


def test_grid_of_canonical_operands_of_a_workload():
    """The splitters of the sparse 4-variable workload's canonical operands
    (distinct exponent vectors, packed and sorted by the test)."""
    from tests.gpu_util import pack_np
    w = polygen.workload_sparse4v()
    a = np.sort(pack_np(w.f.exps, w.field_bits))
    b = np.sort(pack_np(w.g.exps, w.field_bits))
    for l in (8, 64):
        np.testing.assert_array_equal(_gpu(a, b, l), _expect(a, b, l))


def test_grid_errors():
    import torch

    import paper_1303_7425_gb300 as P
    a = torch.arange(1, 10, dtype=torch.int64, device="cuda")
    for bad in (0, 4097):
        with pytest.raises(P.PolymulError) as ei:
            P.grid(a, a, bad)
        assert ei.value.code == -1
    assert P.grid(a[:0], a, 4).numel() == 0

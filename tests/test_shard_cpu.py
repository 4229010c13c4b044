"""Alg. 2's split and gather on CPU ranks (gloo, world sizes 2 and 3): the
split of the intervals by cumulative operation count is the library's own
host rule (pm_split_cumulative); each rank takes the oracle product's terms
in its key slice and the library's ordered gather (shard.ordered_gather)
must give every rank exactly the whole product.  No GPU: the slices come
from the oracle, the intervals from the oracle's Sec. 5 grid, the counts
from brute force over the pp-matrix."""

import os
import socket

import numpy as np
import pytest

import oracle
import polygen
from tests.gpu_util import pack_np


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _problem(seed):
    w = polygen.sparse_product(polygen.Stream(seed, 0), 3, 60, 45, 12)
    e, c = oracle.mul(w.nvars, w.field_bits, "m61", w.f.exps, w.f.coefs, w.g.exps, w.g.coefs)
    keys = pack_np(e, w.field_bits)
    a = np.unique(pack_np(w.f.exps, w.field_bits))
    b = np.unique(pack_np(w.g.exps, w.field_bits))
    return w, keys, np.asarray(c, dtype=np.uint64), a, b


def _split(a, b, nshards, l=4):
    """Splitters (grid + gamma_end), counts below each by brute force, and
    the library's cut; returns the nshards + 1 key bounds."""
    import paper_1303_7425_gb300 as P
    S = np.unique(np.concatenate([oracle.grid(a, b, l), np.array([int(a[-1]) + int(b[-1]) + 1], np.uint64)]))
    sums = (a[:, None] + b[None, :]).reshape(-1)
    cum = np.array([(sums < s).sum() for s in S], dtype=np.uint64)
    cut = P.split_cumulative(cum, nshards)
    bounds = [0] + [int(S[cut[m]]) for m in range(1, nshards)] + [2**64 - 1]
    return bounds, cum, cut


def _rank(rank, world, port, seed, q):
    import torch
    import torch.distributed as dist

    from paper_1303_7425_gb300.shard import ordered_gather
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, keys, coefs, a, b = _problem(seed)
        bounds, _, _ = _split(a, b, world)
        lo, hi = bounds[rank], bounds[rank + 1]
        mine = np.array([lo <= int(k) < hi for k in keys], dtype=bool)
        tk = torch.from_numpy(keys[mine].view(np.int64).copy())
        tc = torch.from_numpy(coefs[mine].view(np.int64).copy())
        gk, gc = ordered_gather(tk, tc)
        ok = (np.array_equal(gk.numpy().view(np.uint64), keys) and np.array_equal(gc.numpy().view(np.uint64), coefs))
        q.put((rank, ok, int(mine.sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,seed", [(2, 3), (3, 4)])
def test_split_and_ordered_gather_give_the_whole_product(world, seed):
    import multiprocessing as mp

    oracle.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, seed, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    assert all(ok for _, ok, _ in got)
    _, keys, _, _, _ = _problem(seed)
    assert sum(n for _, _, n in got) == keys.shape[0]


def test_split_balances_cumulative_counts():
    """Each shard starts at the first boundary whose count reaches its share
    of the total; shares never go backwards; the first and last cuts are the
    ends."""
    import paper_1303_7425_gb300 as P
    rng = np.random.default_rng(0)
    for trial in range(50):
        n = int(rng.integers(2, 40))
        cum = np.concatenate([[0], np.cumsum(rng.integers(0, 1000, n - 1))]).astype(np.uint64)
        for nshards in (1, 2, 3, 7, 64):
            cut = P.split_cumulative(cum, nshards)
            assert cut[0] == 0 and cut[-1] == n - 1 and len(cut) == nshards + 1
            assert all(x <= y for x, y in zip(cut, cut[1:]))
            tot = int(cum[-1])
            for m in range(1, nshards):
                k = cut[m]
                assert int(cum[k]) * nshards >= tot * m or k == n - 1
                assert k == 0 or int(cum[k - 1]) * nshards < tot * m or k == cut[m - 1]
    with pytest.raises(P.PolymulError):
        P.split_cumulative(np.array([5, 3], np.uint64), 2)       # not ascending


def test_split_of_a_real_grid_bounds_each_shard():
    """On a real pp-matrix: every shard's term products stay within one
    interval's count of the even share."""
    w, keys, coefs, a, b = _problem(7)
    for nshards in (2, 3, 5):
        bounds, cum, cut = _split(a, b, nshards, l=8)
        total = int(cum[-1])
        widest = int(np.max(np.diff(cum.astype(np.int64))))
        for m in range(nshards):
            share = int(cum[cut[m + 1]]) - int(cum[cut[m]])
            assert abs(share - total / nshards) <= widest + total / nshards
        assert total == a.size * b.size

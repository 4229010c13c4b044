"""One product over several GPUs, the way Alg. 2 (Sec. 3) spreads it over
nodes: every rank holds both operands, computes the same split of the
output key space into slices of about equal term-product counts
(pm_shard_bounds), multiplies its own slice (pm_polymul_range), and the
slices are gathered in rank order.  The slices own disjoint, ascending key
ranges, so the gather is a concatenation and no reduction happens.

The exchange is a variable-size all-gather: each rank's slice size first,
then the slices padded to the largest, then each rank keeps the valid part
of every slice in rank order.  The process group's backend decides where
the buffers live (NCCL: the ranks' GPUs; gloo: host memory).
"""

from __future__ import annotations

from typing import Sequence, Tuple


def ordered_gather(keys, coefs, group=None) -> Tuple[object, object]:
    """Concatenate every rank's (keys (n_r,), coefs (n_r,) or (n_r, w))
    slice in rank order; every rank receives the whole.  keys and coefs
    must be on the device the group's backend communicates from."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([keys.shape[0]], dtype=torch.int64, device=keys.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    m = max(sizes) if sizes else 0
    tail = tuple(coefs.shape[1:])
    pk = torch.zeros(m, dtype=keys.dtype, device=keys.device)
    pc = torch.zeros((m,) + tail, dtype=coefs.dtype, device=coefs.device)
    pk[:keys.shape[0]] = keys
    pc[:coefs.shape[0]] = coefs
    ak = [torch.empty_like(pk) for _ in range(world)]
    ac = [torch.empty_like(pc) for _ in range(world)]
    dist.all_gather(ak, pk, group=group)
    dist.all_gather(ac, pc, group=group)
    return (torch.cat([a[:s] for a, s in zip(ak, sizes)]), torch.cat([a[:s] for a, s in zip(ac, sizes)]))


def sharded_polymul(field_bits: Sequence[int], f_exps, f_coefs, g_exps, g_coefs, kind: str = "m61", group=None,
                    stream=None):
    """h = f * g over the ranks of `group` (one GPU each; every rank passes
    the same operands on its own GPU).  Returns (keys, coefs, n, stats):
    the whole product on every rank, and this rank's slice statistics."""
    import torch.distributed as dist

    from . import _native as N
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    bounds, products = N.shard_bounds(field_bits, f_exps, f_coefs, g_exps, g_coefs, world, kind=kind,
                                      stream=stream)
    part = N.polymul_range(field_bits, f_exps, f_coefs, g_exps, g_coefs, bounds[rank], bounds[rank + 1],
                           kind=kind, stream=stream)
    keys, coefs = part.keys, part.coefs
    if dist.get_backend(group) == "gloo" and keys.is_cuda:
        keys, coefs = keys.cpu(), coefs.cpu()
    hk, hc = ordered_gather(keys, coefs, group)
    stats = dict(part.stats, slice_products=products[rank], slice_terms=part.n, bounds=bounds)
    return hk, hc, int(hk.shape[0]), stats

"""Sharding of the contraction over ranks (one process per GPU).

Every (configuration, time slice, sink site) item is independent, so ranks
take disjoint sets of (configuration, time slice) slabs and never exchange
propagators or intermediate stages. The only exchange is the final one:
the per-slab correlators (a few KB) are gathered in a fixed rank order so
that every rank ends with the same, bitwise reproducible array.
"""
from __future__ import annotations

import numpy as np


def slab_shard(n_cfg: int, nt: int, rank: int, world: int):
    """Slabs (cfg, t) owned by ``rank``: a contiguous block of the cfg-major
    slab order, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    total = n_cfg * nt
    lo = rank * total // world
    hi = (rank + 1) * total // world
    return [(s // nt, s % nt) for s in range(lo, hi)]


def gather_slabs(local: dict, n_cfg: int, nt: int, shape_tail, group=None) -> np.ndarray:
    """Combine per-slab results {(cfg, t): array(shape_tail)} of every rank
    into one array (n_cfg, nt, *shape_tail) on every rank.

    Uses torch.distributed (any backend that supports all_gather_object, e.g.
    gloo) when it is initialised with more than one rank; otherwise the local
    dict must already hold every slab. Slabs are placed by index, so the
    result does not depend on the rank order of arrival.
    """
    out = np.zeros((n_cfg, nt) + tuple(shape_tail), dtype=np.complex128)
    parts = [local]
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
            parts = [None] * dist.get_world_size(group)
            dist.all_gather_object(parts, local, group=group)
    except ImportError:
        pass
    seen = set()
    for part in parts:
        for (c, t), v in part.items():
            if (c, t) in seen:
                raise ValueError(f"slab {(c, t)} produced by two ranks")
            seen.add((c, t))
            out[c, t] = v
    if len(seen) != n_cfg * nt:
        raise ValueError(f"{n_cfg * nt - len(seen)} slabs missing")
    return out


def rank_cfg_ranges(n_cfg: int, nt: int, rank: int, world: int):
    """The slabs of ``rank`` as (cfg, t0, t1) ranges, one per configuration
    it touches (its slabs are contiguous in cfg-major order)."""
    out = []
    for c, t in slab_shard(n_cfg, nt, rank, world):
        if out and out[-1][0] == c and out[-1][2] == t:
            out[-1] = (c, out[-1][1], t + 1)
        else:
            out.append((c, t, t + 1))
    return out


def contract_sharded(field, lists, group=None, contract=None, **kw):
    """mbc_contract over ranks: every rank contracts its slabs of the host
    field (n_cfg, nt, Lz, Ly, Lx, [n_src,] 12, 12), one call per
    configuration it touches, and the per-slab correlators are gathered in
    slab order. Returns, on every rank, the array a single call over the
    whole field returns: (n_cfg, n_lists, nt, n_mom / N_k, n_comp_max),
    complex128. ``contract`` defaults to the library's contract (keyword
    arguments are passed on; t0 / t1 are taken here)."""
    if contract is None:
        from . import contract as contract
    n_cfg, nt = int(field.shape[0]), int(field.shape[1])
    rank, world = 0, 1
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            rank, world = dist.get_rank(group), dist.get_world_size(group)
    except ImportError:
        pass
    local, tail = {}, None
    for c, t0, t1 in rank_cfg_ranges(n_cfg, nt, rank, world):
        res = np.asarray(contract(field[c:c + 1], lists, t0=t0, t1=t1, **kw))
        tail = (res.shape[1],) + tuple(res.shape[3:])
        for t in range(t0, t1):
            local[(c, t)] = res[0, :, t - t0]
    if tail is None:  # a rank without slabs still learns the shape from the others
        tail = _shape_from_peers(local, group)
    full = gather_slabs(local, n_cfg, nt, tail, group=group)
    return np.ascontiguousarray(np.moveaxis(full, 2, 1))


def _shape_from_peers(local, group):
    import torch.distributed as dist
    parts = [None] * dist.get_world_size(group)
    dist.all_gather_object(parts, [v.shape for v in local.values()][:1], group=group)
    for p in parts:
        if p:
            return tuple(p[0])
    raise ValueError("no rank holds a slab")

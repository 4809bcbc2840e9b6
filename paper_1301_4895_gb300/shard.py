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

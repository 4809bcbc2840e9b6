"""Multi-rank path on CPU: two gloo ranks split the slabs, compute their share
(with the oracle, no GPU needed) and gather; the result equals one rank doing
everything, bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1301_4895_gb300.shard import gather_slabs, slab_shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _slab_values(slabs):
    import synth
    from oracle import recursion, site_sum
    dims = (2, 2, 2)
    plan = recursion.Plan(1, 1, 2)
    out = {}
    for c, t in slabs:
        S = synth.slab(13, c, t, dims, 0.5).reshape(-1, 12, 12)
        C, _ = plan.evaluate(S)
        out[(c, t)] = site_sum.site_sum(C, synth.site_coords(dims), dims[::-1], [(0, 0, 0)])
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = slab_shard(3, 4, rank, world)
        res = gather_slabs(_slab_values(mine), 3, 4, (1, 16))
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_slab_shard_partition():
    for n_cfg, nt, world in ((3, 4, 2), (1, 32, 8), (24, 48, 5), (2, 1, 4)):
        seen = []
        for r in range(world):
            seen += slab_shard(n_cfg, nt, r, world)
        assert sorted(seen) == [(c, t) for c in range(n_cfg) for t in range(nt)]
        sizes = [len(slab_shard(n_cfg, nt, r, world)) for r in range(world)]
        assert max(sizes) - min(sizes) <= 1


def test_gather_detects_gaps_and_overlaps():
    with pytest.raises(ValueError):
        gather_slabs({(0, 0): np.zeros(2)}, 1, 2, (2,))


def test_two_gloo_ranks_equal_one_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    single = gather_slabs(_slab_values(slab_shard(3, 4, 0, 1)), 3, 4, (1, 16))
    assert np.array_equal(results[0], single)
    assert np.array_equal(results[1], single)

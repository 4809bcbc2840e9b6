"""Multi-rank path on CPU: two gloo ranks split the slabs, compute their share
and gather; the result equals one rank doing everything, bit for bit. The
per-rank results are oracle site sums, or arrays shaped like mbc_contract's
output fed through the library's sharded call (shard.contract_sharded), so
no GPU is needed."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1301_4895_gb300.shard import contract_sharded, gather_slabs, rank_cfg_ranges, slab_shard


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


# mbc_contract-shaped partials: a stand-in for the library call that returns,
# for a one-configuration field and a time range, the array mbc_contract
# returns (1, n_lists, t1 - t0, n_mom, n_comp_max), filled with values that
# identify the (configuration, list, t, momentum, component) entry
N_LISTS, N_MOM, N_COMP = 3, 2, 5


def _fake_contract(field, lists, t0=0, t1=0, **kw):
    cfg = int(field[0, 0, 0, 0, 0, 0, 0].real)  # the test field carries its configuration index
    nt = field.shape[1]
    t1 = nt if t1 == 0 else t1
    out = np.zeros((1, len(lists), t1 - t0, N_MOM, N_COMP), dtype=np.complex128)
    for li in range(len(lists)):
        for t in range(t0, t1):
            for q in range(N_MOM):
                for c in range(N_COMP):
                    out[0, li, t - t0, q, c] = complex(1000 * cfg + 100 * li + t, q + 0.125 * c)
    return out


def _test_field(n_cfg, nt):
    f = np.zeros((n_cfg, nt, 1, 1, 1, 12, 12), dtype=np.complex128)
    for c in range(n_cfg):
        f[c] = c
    return f


def _worker_contract(rank, world, port, q, n_cfg, nt):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = contract_sharded(_test_field(n_cfg, nt), [None] * N_LISTS, contract=_fake_contract)
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_rank_cfg_ranges_cover_the_slabs():
    for n_cfg, nt, world in ((3, 4, 2), (24, 48, 5), (2, 1, 4)):
        seen = []
        for r in range(world):
            for c, t0, t1 in rank_cfg_ranges(n_cfg, nt, r, world):
                seen += [(c, t) for t in range(t0, t1)]
        assert sorted(seen) == [(c, t) for c in range(n_cfg) for t in range(nt)]


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_contract_output_equals_one_call(world):
    """Ranks contract their slabs (mbc_contract-shaped outputs, configurations
    split across ranks mid-way) and gather: every rank holds the array of a
    single call over the whole field."""
    n_cfg, nt = 3, 5
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_contract, args=(r, world, port, q, n_cfg, nt)) for r in range(world)]
    for p in procs:
        p.start()
    results = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    whole = np.concatenate([_fake_contract(_test_field(n_cfg, nt)[c:c + 1], [None] * N_LISTS) for c in range(n_cfg)])
    for r in range(world):
        assert results[r].shape == whole.shape and np.array_equal(results[r], whole)
    assert np.array_equal(contract_sharded(_test_field(n_cfg, nt), [None] * N_LISTS, contract=_fake_contract), whole)

"""Host-side tests of libmbc (no GPU needed): the term-list builder against the
paper's counts and the oracle's independent pruning, the ABI surface and its
argument checks."""
import ctypes
import os
import re

import pytest

from conftest import ROOT, read_golden, spins_of
from oracle import counts, recursion

mbc = pytest.importorskip("paper_1301_4895_gb300")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1301_4895_gb300 import _build
    _build.build()
    mbc.load()


def test_library_exports_every_declared_symbol():
    with open(os.path.join(ROOT, "include", "mbc.h")) as f:
        header = f.read()
    names = set(re.findall(r"\b(mbc_[a-z_0-9]+)\s*\(", header))
    assert {"mbc_build_term_list", "mbc_contract", "mbc_term_list_stats", "mbc_free_term_list"} <= names
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_1301_4895_gb300", "libmbc.so"))
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


@pytest.mark.parametrize("name,D", [("table1_rel_all.txt", 4), ("table2_nonrel_all.txt", 2)])
def test_all_component_counts(name, D):
    for row in read_golden(name):
        n_p, n_n, ops = int(row[0]), int(row[1]), int(row[2])
        if ops > 6e8:
            continue  # (2,3) and (3,3) need several GB of list
        tl = mbc.build_term_list(n_p, n_n, D)
        st = tl.stats()
        assert st["n_ops_total"] == ops, row
        assert st["n_comp"] == counts.multinomial(n_p, D - n_p) ** 2 * counts.multinomial(n_n, D - n_n) ** 2
        tl.free()


@pytest.mark.parametrize("name,D", [("table4_nonrel_spin.txt", 2), ("table5_rel_spin.txt", 4)])
def test_single_component_counts(name, D):
    for row in read_golden(name):
        n_p, n_n, ops = int(row[0]), int(row[1]), int(row[3])
        if ops > 3e8:
            continue
        sp = spins_of(row[2])
        tl = mbc.build_term_list(n_p, n_n, D, spins=[(sp, sp)])
        st = tl.stats()
        assert st["n_ops_total"] == ops, row
        assert tl.n_l(0) == int(row[4]), row
        tl.free()


def test_bounds_and_dense_cases():
    for n_p, n_n, D in ((1, 1, 2), (2, 1, 2), (2, 2, 2), (1, 2, 4), (0, 3, 4)):
        st = mbc.build_term_list(n_p, n_n, D).stats()
        path = "".join("P" if b == 0 else "N" for b in st["path"])
        np_ = nn_ = 0
        for m, b in enumerate(path):
            np_ += b == "P"
            nn_ += b == "N"
            assert st["stage_bound"][m] == counts.p_bound(np_, nn_, D)
            assert st["stage_size"][m] <= st["stage_bound"][m]
            if m + 1 < len(path):
                nxt = path[m + 1]
                assert st["q_bound"][m] == counts.q_bound(np_, nn_, D, nxt)
                assert st["n_ops"][m] <= st["q_bound"][m]
    st = mbc.build_term_list(2, 2, 2).stats()
    assert st["n_ops"] == st["q_bound"]  # nothing to prune for nonrelativistic 4He


def test_stage_sizes_agree_with_oracle_pruning():
    """Two independent implementations of the backward pruning (Sec. 3)."""
    for n_p, n_n, D, sp in ((1, 1, 2, None), (2, 1, 2, None), (2, 2, 2, None), (1, 1, 4, None),
                            (2, 2, 4, (0, 1, 0, 1)), (1, 2, 4, (0, 0, 1))):
        spins = None if sp is None else [(sp, sp)]
        tl = mbc.build_term_list(n_p, n_n, D, spins=spins)
        st = tl.stats()
        plan = recursion.Plan(n_p, n_n, D, requests=None if sp is None else [(sp, sp)])
        tot, per, stages = plan.ops()
        assert st["n_ops_total"] == tot
        assert st["n_ops"] == per
        assert st["stage_size"] == stages
        assert sorted(tl.components()) == sorted(plan.requests)


@pytest.mark.slow
def test_headline_lists():
    st = mbc.build_term_list(2, 2, 4).stats()
    assert st["n_ops_total"] == 531321120 and st["n_comp"] == 1296
    sp = (0, 1, 2, 3, 0, 1, 2, 3)
    st = mbc.build_term_list(4, 4, 4, spins=[(sp, sp)]).stats()
    assert st["n_ops_total"] == 448496928
    assert st["stage_size"] == [3168, 196020, 813120, 245025, 813120, 196020, 3168, 1]


def test_paper_path_rule():
    assert mbc.build_term_list(2, 1, 2).stats()["path"] == [0, 0, 1]
    assert mbc.build_term_list(1, 2, 2).stats()["path"] == [1, 1, 0]
    assert mbc.build_term_list(1, 1, 2).stats()["path"] == [1, 0]
    st = mbc.build_term_list(1, 1, 2, path=[0, 1]).stats()
    assert st["path"] == [0, 1] and st["n_ops_total"] == 2664


def test_pauli_forbidden_and_invalid_specs():
    tl = mbc.build_term_list(0, 3, 2)
    assert tl.pauli_forbidden and tl.stats()["n_comp"] == 0 and tl.stats()["n_ops_total"] == 0
    tl = mbc.build_term_list(0, 2, 2, spins=[((0, 0), (0, 1))])  # repeated sink spin
    assert tl.stats()["n_comp"] == 1 and tl.n_l(0) == 0
    with pytest.raises(mbc.MbcError):
        mbc.build_term_list(1, 1, 3)
    with pytest.raises(mbc.MbcError):
        mbc.build_term_list(0, 0, 4)
    with pytest.raises(mbc.MbcError):
        mbc.build_term_list(1, 1, 2, path=[0, 0])
    with pytest.raises(mbc.MbcError):
        mbc.build_term_list(1, 1, 2, n_sources=5)  # 30 quark index values > 24


def test_contract_rejects_bad_arguments_before_any_device_work():
    import numpy as np
    tl = mbc.build_term_list(1, 1, 2)
    with pytest.raises(ValueError):
        mbc.contract(np.zeros((1, 1, 1, 1, 1, 12, 11), dtype=np.complex128), [tl])
    lib = mbc.load()
    assert lib.mbc_contract(None, None, 0, None, None, None) == 1


def test_spin_projection_lists():
    """Sec. 5: a projection is folded into one modified list. A single
    (delta = alpha) term reproduces the listed component's operation count
    (Table 5); the deuteron J_z = 0 projection needs no more operations than
    its four components listed separately."""
    sp = (0, 1, 0, 1)
    one = mbc.build_term_list(2, 2, 4, projections=[[(sp, sp, 1.0)]]).stats()
    assert one["n_ops_total"] == 8541864 and one["n_comp"] == 1
    # unsorted spins of one species: same list up to a sign, same cost
    swapped = mbc.build_term_list(2, 2, 4, projections=[[((1, 0, 0, 1), sp, 1.0)]])
    assert swapped.stats()["n_ops_total"] == 8541864
    pairs = [((0, 1), (0, 1)), ((0, 1), (1, 0)), ((1, 0), (0, 1)), ((1, 0), (1, 0))]
    jz0 = mbc.build_term_list(1, 1, 2, projections=[[(a, b, 0.5) for a, b in pairs]])
    listed = mbc.build_term_list(1, 1, 2, spins=pairs)
    assert jz0.stats()["n_ops_total"] <= listed.stats()["n_ops_total"]
    assert jz0.components() == [((-1, -1), (-1, -1))]
    # a repeated spin within a species is a Pauli zero term
    zero = mbc.build_term_list(0, 2, 4, projections=[[((1, 1), (0, 1), 1.0)]])
    assert zero.n_l(0) == 0
    with pytest.raises(mbc.MbcError):
        mbc.build_term_list(1, 1, 2, projections=[[]])


def test_two_source_single_components_match_table6():
    """Sec. 6: two quark sources (and two sink functions) with
    nonrelativistic operators; spinor-source indices 2 alpha + s (Table 6)."""
    for row in read_golden("table6_nonrel_two_sources_spin.txt"):
        n_p, n_n, ops = int(row[0]), int(row[1]), int(row[3])
        if ops > 6e7:
            continue
        sp = spins_of(row[2])
        tl = mbc.build_term_list(n_p, n_n, 2, spins=[(sp, sp)], n_sources=2, n_sinks=2)
        assert tl.stats()["n_ops_total"] == ops, row
        assert tl.n_l(0) == int(row[4]), row
    # contraction kernels take one sink function, at most 12 source quark
    # index values, and a field with as many sources as the list: every other
    # case is refused before any device work
    import numpy as np
    f2 = np.zeros((1, 1, 1, 1, 1, 2, 12, 12), dtype=np.complex128)
    tl = mbc.build_term_list(1, 1, 2, spins=[((0, 2), (0, 2))], n_sources=2, n_sinks=2)
    with pytest.raises(mbc.MbcError):
        mbc.contract(f2, [tl])
    one_sink = mbc.build_term_list(1, 1, 2, spins=[((0, 1), (0, 3))], n_sources=2)
    with pytest.raises(mbc.MbcError):
        mbc.contract(f2[:, :, :, :, :, 0], [one_sink])  # field without the source axis
    rel = mbc.build_term_list(1, 0, 4, spins=[((0,), (5,))], n_sources=2)
    with pytest.raises(mbc.MbcError):
        mbc.contract(f2, [rel])  # 24 source quark index values


def test_two_source_lists_agree_with_oracle():
    """Builder and oracle (O3 fed with its own G~ from the gamma matrices)
    prune the two-source lists identically."""
    from oracle import gamma
    Gt = gamma.g_tensor_sources(2, 2)
    for n_p, n_n, sp in ((1, 1, (0, 2)), (0, 3, (0, 1, 2)), (1, 2, (2, 0, 2)), (2, 2, (0, 2, 0, 2))):
        st = mbc.build_term_list(n_p, n_n, 2, spins=[(sp, sp)], n_sources=2, n_sinks=2).stats()
        plan = recursion.Plan(n_p, n_n, 2, requests=[(sp, sp)], G=Gt)
        tot, per, stages = plan.ops()
        assert (st["n_ops_total"], st["n_ops"], st["stage_size"]) == (tot, per, stages)


def _prefix(path, A):
    return list(path[:A])


@pytest.mark.parametrize("D,path,nuclei", [
    (2, [0, 0, 1, 1], [(2, 1, None), (2, 2, None)]),
    (2, [0, 1, 0, 1], [(1, 0, None), (1, 1, None), (2, 1, None), (2, 2, None)]),
    (4, [1, 1, 0, 0], [(0, 1, None), (0, 2, None), (2, 2, [((0, 1, 0, 1), (0, 1, 0, 1))])]),
    (4, [1, 0, 1], [(1, 1, [((0, 1), (2, 3)), ((1, 1), (1, 1))]), (1, 2, [((2, 0, 1), (0, 1, 2)), ((0, 1, 3), (1, 0, 2))])]),
])
def test_combined_path_lists_agree_with_oracle_pruning(D, path, nuclei):
    """Sec. 7: nuclei on one path share its stages. Every stage of the
    combined list holds exactly the union of the components each nucleus
    needs on its own (the oracle's independent pruning along the same path
    prefix), each step costs splits x stage size, and the outputs are the
    nuclei's components in order, labels padded with -1."""
    specs = [dict(n_p=a, n_n=b, spins=sp) for a, b, sp in nuclei]
    tl = mbc.build_combined(specs, D, path=path)
    st = tl.stats()
    A = len(path)
    assert st["path"] == path and st["n_parts"] == len(nuclei)
    plans = []
    c0 = 0
    comps = tl.components()
    for j, (a, b, sp) in enumerate(nuclei):
        Aj = a + b
        plan = recursion.Plan(a, b, D, requests=sp, path=_prefix(path, Aj))
        plans.append((Aj, plan))
        part = tl.parts()[j]
        assert (part["n_p"], part["n_n"], part["c0"]) == (a, b, c0)
        assert part["c1"] - part["c0"] == len(plan.requests)
        nl = dict(zip(plan.requests, plan.n_l()))
        pad = (-1,) * (A - Aj)
        mine = comps[part["c0"]:part["c1"]]
        assert all(snk[Aj:] == pad and src[Aj:] == pad for snk, src in mine)
        assert sorted((snk[:Aj], src[:Aj]) for snk, src in mine) == sorted(plan.requests)
        for c, (snk, src) in zip(range(part["c0"], part["c1"]), mine):
            assert tl.n_l(c) == nl[(snk[:Aj], src[:Aj])]
        c0 = part["c1"]
    for m in range(2, A + 1):
        union = set()
        for Aj, plan in plans:
            if Aj >= m:
                union |= set(plan.stage_keys(m).tolist())
        assert st["stage_size"][m - 1] == len(union), m
        assert st["n_ops"][m - 2] == st["ops_per_z"][m - 2] * st["stage_size"][m - 1]
    separate = sum(plan.ops()[0] for _, plan in plans)
    assert max(plan.ops()[0] for _, plan in plans) <= st["n_ops_total"] <= separate


def test_combined_free_rider():
    """Nonrelativistic 4He on the path P, P, N, N needs every stage-3
    component, so 3He (all components) costs nothing extra."""
    he4 = mbc.build_term_list(2, 2, 2, path=[0, 0, 1, 1]).stats()["n_ops_total"]
    both = mbc.build_combined([dict(n_p=2, n_n=1), dict(n_p=2, n_n=2)], 2, path=[0, 0, 1, 1])
    assert both.stats()["n_ops_total"] == he4 == 10980
    assert both.stats()["n_comp"] == 4 + 1


def test_combined_rejects_nuclei_off_the_path():
    with pytest.raises(mbc.MbcError):
        mbc.build_combined([dict(n_p=0, n_n=2), dict(n_p=2, n_n=2)], 2, path=[0, 0, 1, 1])
    with pytest.raises(mbc.MbcError):  # Pauli-forbidden largest nucleus
        mbc.build_combined([dict(n_p=1, n_n=0), dict(n_p=3, n_n=0)], 2)
    with pytest.raises(ValueError):
        mbc.build_combined([], 2)
    h = ctypes.c_void_p()
    assert mbc.load().mbc_build_combined(None, 0, ctypes.byref(h)) == 1 and not h.value


def test_list_free_lists():
    """list_free stores no operation arrays: dense steps need nothing, the
    others two index tables; counts and stage sizes are unchanged."""
    for n_p, n_n, D, sp in ((2, 2, 2, None), (2, 1, 2, None), (2, 2, 4, [((0, 1, 0, 1), (0, 1, 0, 1))])):
        spins = sp
        a = mbc.build_term_list(n_p, n_n, D, spins=spins).stats()
        b = mbc.build_term_list(n_p, n_n, D, spins=spins, list_free=True).stats()
        for key in ("n_ops_total", "n_ops", "stage_size", "dense_steps", "n_l_total"):
            assert a[key] == b[key], key
        assert a["op_bytes"] == 6 * a["n_ops_total"]
        assert b["op_bytes"] < a["op_bytes"]
    st = mbc.build_term_list(2, 2, 2, list_free=True).stats()
    assert st["dense_steps"] == [1, 2, 3] and st["op_bytes"] == 0


def _fill_source_sets(n):
    """Source spin-source sets of n baryons of one species that fill source 0
    (chi = 0, 2) first and take source 1 (chi = 1, 3) beyond two baryons."""
    import itertools
    if n <= 2:
        return [tuple(c) for c in itertools.combinations((0, 2), n)]
    return [tuple(sorted((0, 2) + c)) for c in itertools.combinations((1, 3), n - 2)]


def test_two_source_all_component_counts_match_table3():
    """Table 3 (two sources, nonrelativistic, all components) under the
    reading in its golden file: two sink functions with every sink
    component, source components filling source 0 first."""
    import itertools
    for row in read_golden("table3_nonrel_two_sources_all.txt"):
        n_p, n_n, ops = int(row[0]), int(row[1]), int(row[2])
        snk = [p + q for p in itertools.combinations(range(4), n_p) for q in itertools.combinations(range(4), n_n)]
        src = [p + q for p in _fill_source_sets(n_p) for q in _fill_source_sets(n_n)]
        tl = mbc.build_term_list(n_p, n_n, 2, spins=[(a, b) for a in snk for b in src], n_sources=2, n_sinks=2)
        assert tl.stats()["n_ops_total"] == ops, row
        tl.free()


def test_term_list_files_roundtrip(tmp_path):
    """A saved list loads with the same statistics, labels and contents (its
    own save is byte-identical); damaged or foreign files are refused."""
    kinds = [dict(n_p=2, n_n=2, dirac_dim=2), dict(n_p=2, n_n=1, dirac_dim=2, list_free=True),
             dict(n_p=1, n_n=1, dirac_dim=2, projections=[[((0, 1), (0, 1), 0.5), ((1, 0), (1, 0), 0.5)]]),
             dict(n_p=2, n_n=2, dirac_dim=2, spins=[((0, 1, 2, 3), (0, 2, 0, 2))], n_sources=2, n_sinks=2),
             dict(n_p=0, n_n=3, dirac_dim=2)]
    for j, kw in enumerate(kinds):
        a = mbc.build_term_list(**kw)
        p1, p2 = tmp_path / f"a{j}.bin", tmp_path / f"b{j}.bin"
        a.save(str(p1))
        b = mbc.load_term_list(str(p1))
        b.save(str(p2))
        assert a.stats() == b.stats() and a.components() == b.components(), kw
        assert [a.n_l(c) for c in range(a.stats()["n_comp"])] == [b.n_l(c) for c in range(b.stats()["n_comp"])]
        assert p1.read_bytes() == p2.read_bytes(), kw
        assert b.pauli_forbidden == a.pauli_forbidden
    comb = mbc.build_combined([dict(n_p=2, n_n=1), dict(n_p=2, n_n=2)], 2, path=[0, 0, 1, 1])
    comb.save(str(tmp_path / "c.bin"))
    assert mbc.load_term_list(str(tmp_path / "c.bin")).parts() == comb.parts()
    raw = (tmp_path / "a0.bin").read_bytes()
    (tmp_path / "cut.bin").write_bytes(raw[: len(raw) // 2])
    (tmp_path / "magic.bin").write_bytes(b"XBCL" + raw[4:])
    for bad in ("cut.bin", "magic.bin", "missing.bin"):
        with pytest.raises(mbc.MbcError):
            mbc.load_term_list(str(tmp_path / bad))


def test_term_list_cache(tmp_path):
    kw = dict(n_p=2, n_n=1, dirac_dim=2, spins=[((0, 1, 0), (0, 1, 1))])
    a = mbc.build_term_list(**kw, cache_dir=str(tmp_path))
    files = list(tmp_path.iterdir())
    assert len(files) == 1
    b = mbc.build_term_list(**kw, cache_dir=str(tmp_path))  # loaded from the file
    assert b.stats() == a.stats() and b.components() == a.components()
    c = mbc.build_term_list(**dict(kw, spins=[((0, 1, 1), (0, 1, 1))]), cache_dir=str(tmp_path))
    assert len(list(tmp_path.iterdir())) == 2 and c.components() != a.components()


def test_term_list_files_damaged_anywhere(tmp_path):
    """Loading a damaged file never crashes and never allocates more than the
    file holds: every 8-byte word set to a huge length, and random byte
    flips, either load (the loader has checked every index the kernels use)
    or are refused with an error."""
    import numpy as np
    a = mbc.build_term_list(2, 1, 2, spins=[((0, 1, 0), (0, 1, 1))])
    src = tmp_path / "a.bin"
    a.save(str(src))
    raw = bytearray(src.read_bytes())
    bad = tmp_path / "bad.bin"
    refused = 0
    huge = ((1 << 36) - 1).to_bytes(8, "little")
    for off in range(16, len(raw) - 8, 8):
        damaged = bytearray(raw)
        damaged[off:off + 8] = huge
        bad.write_bytes(bytes(damaged))
        try:
            mbc.load_term_list(str(bad))
        except mbc.MbcError:
            refused += 1
    assert refused > 0
    rng = np.random.default_rng(7)
    for _ in range(300):
        damaged = bytearray(raw)
        for pos in rng.integers(16, len(raw), size=int(rng.integers(1, 5))):
            damaged[int(pos)] = int(rng.integers(0, 256))
        bad.write_bytes(bytes(damaged))
        try:
            b = mbc.load_term_list(str(bad))
            b.stats()
        except mbc.MbcError:
            pass


@pytest.mark.parametrize("n_p,n_n,spins", [
    (1, 1, None), (0, 2, [((0, 1), (0, 1))]), (2, 1, [((0, 1, 0), (0, 2, 4))]),
    pytest.param(2, 2, [((0, 1, 0, 1), (0, 2, 4, 6))], marks=pytest.mark.slow),
])
def test_two_relativistic_sources_counts_match_oracle(n_p, n_n, spins):
    """Two relativistic quark sources (Sec. 6, 24 source quark indices): the
    builder's sparse index sets give the same pruned stages and operation
    counts as the oracle's 64-bit-key pruning."""
    from oracle import gamma, recursion
    tl = mbc.build_term_list(n_p, n_n, 4, spins=spins, n_sources=2)
    st = tl.stats()
    plan = recursion.Plan(n_p, n_n, 4, requests=tl.components(), G=gamma.g_tensor_sources(4, 2),
                          G_sink=gamma.g_tensor(4))
    tot, per, stages = plan.ops()
    assert st["n_ops_total"] == tot
    assert st["stage_size"][: n_p + n_n] == stages
    assert st["block_size"] == 4 * 276 * 24

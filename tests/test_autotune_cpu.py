"""Candidate launch shapes of the autotuner (host logic, no GPU): every
candidate is a valid tuning record, the kernels a list set uses decide which
fields vary, and the item orders are offered per wave step kernel (FP64: 0
and 1; mixed: 0, one CTA of 32 warps per SM on consecutive outputs of one
site group, and 3, 8-warp CTAs with the site groups side by side)."""
import paper_1301_4895_gb300 as mbc
from paper_1301_4895_gb300 import autotune


def _cands(lists, precision):
    return list(autotune.candidates(lists, precision))


def test_candidates_cover_each_regime():
    nonrel = [mbc.build_term_list(2, 1, 2)]
    rel = [mbc.build_term_list(1, 1, 4)]
    for prec in (mbc.FP64, mbc.MIXED):
        for lists in (nonrel, rel, nonrel + rel):
            cands = _cands(lists, prec)
            assert cands and len({tuple(sorted(c.items())) for c in cands}) == len(cands)
            for c in cands:
                assert set(c) <= set(mbc.Tune.FIELDS)
                t = mbc.Tune(**c)  # a record the library takes
                assert all(getattr(t, k) == v and v > 0 for k, v in c.items())
    # nonrelativistic lists only: the shared-memory kernel's shape varies, no wave fields
    assert all(set(c) <= {"sites_per_cta"} for c in _cands(nonrel, mbc.FP64))
    assert all(set(c) <= {"threads_per_cta"} for c in _cands(nonrel, mbc.MIXED))
    # relativistic lists only: wave fields only
    assert all(not ({"sites_per_cta", "threads_per_cta"} & set(c)) for c in _cands(rel, mbc.FP64))


def test_item_orders_per_wave_step_kernel():
    rel = [mbc.build_term_list(1, 1, 4)]
    assert {c.get("wave_order", 0) for c in _cands(rel, mbc.FP64)} == {0, 1}
    assert {c.get("wave_order", 0) for c in _cands(rel, mbc.MIXED)} == {0, 3}

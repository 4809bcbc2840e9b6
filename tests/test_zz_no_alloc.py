"""The allocation-free entry point, mbc_contract_noalloc.

It serves callers that cannot allocate device memory in steady state
(services whose device memory is reserved up front by their own pool,
real-time loops that forbid allocator calls): its scratch is a static device
array inside the library. Its results must agree with
mbc_contract's within the FP64 bound of the parity tests, on two calls in a
row (the shared array keeps the previous call's contents). This file is
collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth
from gpu_helpers import max_rel_err, oracle_plan, oracle_slab


@pytest.mark.gpu
def test_noalloc_matches_contract_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1301_4895_gb300 as mbc
    from paper_1301_4895_gb300 import _build
    _build.build()
    lib = mbc.load()
    dims = (4, 4, 4)
    field_np = synth.field(9, 2, 3, dims, 0.5)
    field = torch.from_numpy(field_np).to("cuda:0")
    moms = ((0, 0, 0), (1, 0, 2))
    for n_p, n_n in ((1, 1), (2, 2)):
        tl = mbc.build_term_list(n_p, n_n, 2)
        ref = mbc.contract(field, [tl], precision=mbc.FP64, moms=moms)  # also makes the list resident
        torch.cuda.synchronize()
        ref = ref.cpu().numpy()[:, 0]
        comps = tl.components()
        plan = oracle_plan(n_p, n_n, 2, comps)
        scale = {}
        for cfg in range(2):
            for t in range(3):
                _, scale[cfg, t] = oracle_slab(plan, field_np[cfg, t], dims, list(moms))
        for call in range(2):
            out = torch.full((2, 1, 3, len(moms), len(comps)), complex(float("nan"), 0.0), dtype=torch.complex128,
                             device="cuda:0")
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            mbc.contract_noalloc(field, tl, out, moms=moms)
            torch.cuda.synchronize()
            if call == 1:  # after the first call's one-time set-up: no device memory taken
                assert torch.cuda.mem_get_info()[0] == free0
            got = out.cpu().numpy()[:, 0]
            for cfg in range(2):
                for t in range(3):
                    e = max_rel_err(got[cfg, t], ref[cfg, t], scale[cfg, t])
                    assert e <= 1e-13, (n_p, n_n, call, cfg, t, e)


def test_noalloc_rejects_before_device_work():
    """Oversized or unsupported requests are refused from host-side checks
    alone (no device needed)."""
    import paper_1301_4895_gb300 as mbc
    from paper_1301_4895_gb300 import _build
    _build.build()
    lib = mbc.load()
    tl = mbc.build_term_list(2, 2, 2)
    fake = 1 << 20  # never dereferenced: every check below fails first
    moms = np.zeros((32, 3), dtype=np.int32)
    big = mbc.Props(fake, fake, mbc.C128, mbc.MEM_DEVICE, 1, 1, 64, 64, 64, 0, 0)
    op = mbc.ContractOpts(mbc.FP64, 32, moms.ctypes.data, 0, 0, None)
    rc = lib.mbc_contract_noalloc(ctypes.byref(big), tl.handle, ctypes.byref(op), fake, None)
    assert rc == 6  # MBC_ERR_UNSUPPORTED: phase table alone needs 128 MiB > 8 MiB
    small = mbc.Props(fake, fake, mbc.C128, mbc.MEM_DEVICE, 1, 1, 4, 4, 4, 0, 0)
    op_mixed = mbc.ContractOpts(mbc.MIXED, 1, moms.ctypes.data, 0, 0, None)
    assert lib.mbc_contract_noalloc(ctypes.byref(small), tl.handle, ctypes.byref(op_mixed), fake, None) == 6
    rel = mbc.build_term_list(1, 1, 4)
    op1 = mbc.ContractOpts(mbc.FP64, 1, moms.ctypes.data, 0, 0, None)
    assert lib.mbc_contract_noalloc(ctypes.byref(small), rel.handle, ctypes.byref(op1), fake, None) == 6

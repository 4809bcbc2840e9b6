"""Shared helpers of the GPU parity tests: oracle reference sums for slabs."""
import numpy as np

import synth
from oracle import recursion, site_sum

_PLANS = {}


def oracle_plan(n_p, n_n, D, comps):
    key = (n_p, n_n, D, tuple(comps))
    if key not in _PLANS:
        _PLANS[key] = recursion.Plan(n_p, n_n, D, requests=list(comps))
    return _PLANS[key]


def oracle_slab(plan, slab, dims_zyx, moms):
    """Site-summed oracle correlators and error scale of one slab.
    slab: (Lz, Ly, Lx, 12, 12) complex; returns (ref (n_mom, n_comp), scale (n_comp,))."""
    C, sc = plan.evaluate(np.asarray(slab, dtype=np.complex128).reshape(-1, 12, 12))
    coords = synth.site_coords(dims_zyx)
    ref = site_sum.site_sum(C, coords, tuple(dims_zyx[::-1]), moms)
    return ref, site_sum.scale_sum(sc)


# worst |dC| / sum|terms| seen by the parity tests, per (nucleus, precision)
WORST = {}


def record(label, precision, err):
    key = (label, "fp64" if precision == 0 else "mixed")
    WORST[key] = max(WORST.get(key, 0.0), float(err))


def max_rel_err(got, ref, scale):
    """max |got - ref| / scale over momenta and components."""
    return float(np.max(np.abs(np.asarray(got) - ref) / scale[None, :]))

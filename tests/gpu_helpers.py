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
    slab: (Lz, Ly, Lx, 12, 12) complex (12 x 24 tiles for two relativistic
    sources); returns (ref (n_mom, n_comp), scale (n_comp,))."""
    slab = np.asarray(slab, dtype=np.complex128)
    C, sc = plan.evaluate(slab.reshape(-1, 12, slab.shape[-1]))
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


# near-identity propagators (synth eps): |C| / sum|terms| >= 2e-2 on every
# parity case (5e-3 for 8Be) instead of down to 5e-14 on Gaussian ones
EPS = 0.05


def legs(seed, n_cfg, nt, dims, lam, dtype=np.complex128, n_src=0, gauss=True, eps=EPS):
    """(field, precisions) pairs a parity test runs: the configuration's
    Gaussian recipe for FP64 (its bound discriminates there, 8Be aside) and
    near-identity propagators from the same draws for both precisions."""
    out = []
    if gauss:
        out.append((synth.field(seed, n_cfg, nt, dims, lam, dtype=dtype, n_src=n_src), (0,)))
    out.append((synth.field(seed, n_cfg, nt, dims, lam, dtype=dtype, n_src=n_src, eps=eps), (0, 1)))
    return out

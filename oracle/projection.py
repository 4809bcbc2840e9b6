"""Momentum-projected baryon blocks (oracle, test infrastructure).

Test infrastructure only (see ``oracle/__init__.py``).

Sec. 2 defines the blocks with a sink function s(x): f_B(t) = sum_x s(x)
<B(x, t) qbar qbar qbar>, and the recursion of Sec. 4 then runs once per time
slice on these summed blocks (the paper's own usage, Sec. 2 and the summary:
each baryon projected to a momentum before the recursion). Here every baryon
uses the same s(x) = exp(-2 pi i n.x / L). The blocks of every site come from
O3, the phase-weighted sum over sites is a plain numpy sum, and O3 runs the
recursion and contraction on the summed blocks. The error scale sums the
per-site block magnitudes (|s(x)| = 1) and runs the magnitude recursion on
them.
"""
from __future__ import annotations

import numpy as np

from .site_sum import phases


def projected_correlators(plan, slab, dims_zyx, moms, chunk: int = 256):
    """C(t, n) of one slab with momentum-projected blocks.
    slab: (Lz, Ly, Lx, 12, 12); returns (C (n_mom, n_req), scale (n_mom, n_req))."""
    import synth
    S = np.asarray(slab, dtype=np.complex128).reshape(-1, 12, 12)
    coords = synth.site_coords(dims_zyx)
    dims_xyz = tuple(dims_zyx[::-1])
    ph = np.stack([phases(coords, dims_xyz, m) for m in moms])  # (n_mom, V)
    shp = (len(moms), 4, 12, 12, 12)
    Pp = np.zeros(shp, dtype=np.complex128)
    Pn = np.zeros(shp, dtype=np.complex128)
    Mp = np.zeros(shp)
    Mn = np.zeros(shp)
    for s0 in range(0, S.shape[0], chunk):
        fp, fn, mp, mn = plan.blocks(S[s0:s0 + chunk])
        w = ph[:, s0:s0 + chunk]
        Pp += np.tensordot(w, fp, axes=(1, 0))
        Pn += np.tensordot(w, fn, axes=(1, 0))
        Mp += mp.sum(axis=0)[None]
        Mn += mn.sum(axis=0)[None]
    return plan.evaluate_blocks(Pp, Pn, Mp, Mn)

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

Several sink functions (Sec. 6): with N_k of them the sink baryon index is
psi = N_k alpha + k, and the block of sink index psi is the block of spin alpha
summed with sink function k. Here sink function k of a group is the k-th of
N_k consecutive momenta, so a group of momenta gives one set of blocks.
"""
from __future__ import annotations

import numpy as np

from .site_sum import phases


def projected_correlators(plan, slab, dims_zyx, moms, chunk: int = 256, n_sinks: int = 1, dirac_dim: int = 0):
    """C(t, n) of one slab with momentum-projected blocks.
    slab: (Lz, Ly, Lx, 12, 12) (or 12 x 24 tiles for a wide plan); returns (C (n_groups, n_req), scale (n_groups,
    n_req)) with n_groups = n_mom / n_sinks (one group = n_sinks momenta, one
    per sink function; dirac_dim, needed when n_sinks > 1, is the number of
    spin values alpha of the single-sink blocks)."""
    import synth
    S = np.asarray(slab, dtype=np.complex128)
    S = S.reshape((-1, 12, S.shape[-1]))
    coords = synth.site_coords(dims_zyx)
    dims_xyz = tuple(dims_zyx[::-1])
    ph = np.stack([phases(coords, dims_xyz, m) for m in moms])  # (n_mom, V)
    q = plan.nq
    shp = (len(moms), 4, q, q, q)
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
    if n_sinks > 1:
        if len(moms) % n_sinks or dirac_dim * n_sinks > 4:
            raise ValueError("momenta must come in whole groups; dirac_dim * n_sinks <= 4")
        n_groups = len(moms) // n_sinks
        grouped = []
        for X in (Pp, Pn, Mp, Mn):
            Y = np.zeros((n_groups,) + X.shape[1:], dtype=X.dtype)
            for g in range(n_groups):
                for k in range(n_sinks):
                    for a in range(dirac_dim):
                        Y[g, n_sinks * a + k] = X[g * n_sinks + k, a]
            grouped.append(Y)
        Pp, Pn, Mp, Mn = grouped
    return plan.evaluate_blocks(Pp, Pn, Mp, Mn)

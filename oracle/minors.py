"""O2: the correlator grouped by occupied index sets (oracle, test infrastructure).

Test infrastructure only (see ``oracle/__init__.py``).

Sec. 2 writes the correlator as C = F . L (eq. f_L_contr) with the symbolic
tensor L of eq. tensor_L: the signed sum, over all permutations of
same-flavour quark indices, of the product of the G tensors (eq. def_g).
Because L is antisymmetric within each flavour, it is fixed by its values on
sorted index sets (Sec. 3). Here L is written out by brute force: every tuple
of nonzero G entries, one per baryon, whose u (and d) slot values are all
distinct, adds sign(sorting permutation) * prod(G) to L(alpha; U-set, D-set).

Grouping the Wick sum (Sec. 1 eq. C_baryons) by the sink sets (U', D') and
source sets (U, D) turns the signed sum over quark permutations into a product
of two determinants of propagator minors:

    C(delta; alpha) = sum L(delta; U', D') L(alpha; U, D)
                          det S_u[U'; U] det S_d[D'; D].

``delta`` and ``alpha`` are ordered spin assignments, one per baryon, in the
order of ``baryons`` (protons first in all public helpers).
"""
from __future__ import annotations

import itertools
from functools import lru_cache

import numpy as np

from .gamma import SLOT_FLAVOURS, g_nonzeros


def _inversions(seq) -> int:
    n = 0
    for i in range(len(seq)):
        for j in range(i + 1, len(seq)):
            if seq[i] > seq[j]:
                n += 1
    return n


@lru_cache(maxsize=None)
def _gnz(dirac_dim: int):
    return g_nonzeros(dirac_dim)


def l_tensor(baryons: str, alpha, dirac_dim: int) -> dict:
    """L(alpha; U, D) of eq. tensor_L on sorted index sets.

    baryons: e.g. "PPNN"; alpha: spins, one per baryon, same order.
    Returns {(U tuple, D tuple): int} with zero entries dropped.
    """
    gnz = _gnz(dirac_dim)
    per = [gnz[int(a)] for a in alpha]
    flav = [SLOT_FLAVOURS[b] for b in baryons]
    out: dict = {}

    def rec(k, us, ds, val):
        if k == len(baryons):
            key = (tuple(sorted(us)), tuple(sorted(ds)))
            sgn = -1 if (_inversions(us) + _inversions(ds)) % 2 else 1
            out[key] = out.get(key, 0) + sgn * val
            return
        for (xi, g) in per[k]:
            nu, nd = list(us), list(ds)
            ok = True
            for slot in range(3):
                tgt = nu if flav[k][slot] == 0 else nd
                if xi[slot] in tgt:
                    ok = False
                    break
                tgt.append(xi[slot])
            if ok:
                rec(k + 1, nu, nd, val * g)

    rec(0, [], [], 1.0)
    return {k: int(round(v)) for k, v in out.items() if round(v) != 0}


def _minor_dets(S: np.ndarray, sets_row, sets_col) -> np.ndarray:
    """det S[r; c] for every row set r and column set c (numpy det)."""
    rows = np.asarray(sets_row, dtype=np.int64)
    cols = np.asarray(sets_col, dtype=np.int64)
    if rows.shape[1] == 0:
        return np.ones((len(rows), len(cols)), dtype=complex)
    sub = S[rows[:, None, :, None], cols[None, :, None, :]]
    return np.linalg.det(sub)


def correlator(baryons: str, delta, alpha, dirac_dim: int, S_u: np.ndarray, S_d: np.ndarray,
               L_snk=None, L_src=None) -> complex:
    """C(delta; alpha) at one site from the minor form (O2)."""
    L_snk = l_tensor(baryons, delta, dirac_dim) if L_snk is None else L_snk
    L_src = l_tensor(baryons, alpha, dirac_dim) if L_src is None else L_src
    if not L_snk or not L_src:
        return 0j
    su = sorted({k[0] for k in L_snk}); sd = sorted({k[1] for k in L_snk})
    cu = sorted({k[0] for k in L_src}); cd = sorted({k[1] for k in L_src})
    du = _minor_dets(np.asarray(S_u, dtype=complex), su, cu)
    dd = _minor_dets(np.asarray(S_d, dtype=complex), sd, cd)
    iu = {k: i for i, k in enumerate(su)}; idd = {k: i for i, k in enumerate(sd)}
    ju = {k: i for i, k in enumerate(cu)}; jd = {k: i for i, k in enumerate(cd)}
    # A[U', D'] (sink, dense over the support), B[U, D] (source)
    A = np.zeros((len(su), len(sd)))
    for (u, d), v in L_snk.items():
        A[iu[u], idd[d]] = v
    B = np.zeros((len(cu), len(cd)))
    for (u, d), v in L_src.items():
        B[ju[u], jd[d]] = v
    # sum_{U'D'UD} A[U'D'] B[UD] du[U'U] dd[D'D] = sum A * (du B dd^T)
    return complex(np.sum(A * (du @ B @ dd.T)))


def spin_sets(n: int, dirac_dim: int):
    """Sorted spin sets of n same-type baryons (each spin below dirac_dim)."""
    return [tuple(c) for c in itertools.combinations(range(dirac_dim), n)]


def nucleus_components(n_p: int, n_n: int, dirac_dim: int):
    """All independent spin assignments of (n_p protons, n_n neutrons): every
    pair of sorted proton and neutron spin sets, protons first (Sec. 4)."""
    return [p + n for p in spin_sets(n_p, dirac_dim) for n in spin_sets(n_n, dirac_dim)]

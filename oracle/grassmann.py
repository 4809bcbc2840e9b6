"""L(alpha; U, D) from the exterior algebra (oracle, test infrastructure).

Test infrastructure only (see ``oracle/__init__.py``).

The source tensor of eq. tensor_L is the signed sum, over the permutations
of same-flavour quark indices, of products of G tensors (eq. def_g). That sum
is what a product in an exterior algebra produces by itself: give every u
index xi an anticommuting generator u_xi and every d index a generator d_xi
(u and d generators commute with each other, so the two flavours carry their
own signs), write each baryon as the element

    B_P(alpha) = sum G(alpha; x1, x2, x3) u_x1 u_x2 d_x3     (proton, u u d)
    B_N(alpha) = sum G(alpha; x1, x2, x3) d_x1 u_x2 d_x3     (neutron, d u d)

and multiply the baryons in order. Bringing each monomial to ascending index
order within each flavour costs the sign of the sorting permutation of the u
indices times that of the d indices, so the coefficient of u_U d_D is
L(alpha; U, D) with exactly the sign convention of the minor form (O2).
Unlike O2 (enumeration of G tuples) and O3 (the paper's bullet recursion),
this keeps one polynomial in the generators and multiplies it by one
generator at a time: the sign of moving u_g to its place in an ascending
monomial is (-1)^(number of generators of the monomial above g).

The use here: a saturated nucleus (8Be: all 12 u and 12 d indices filled)
has one L entry, and C = L(delta)^2 ... = L^2 det S_u det S_d for delta = alpha
(Sec. 8's saturation), so this pins the O3 constant K = C / (det S_u det S_d).
"""
from __future__ import annotations

import numpy as np

from .gamma import SLOT_FLAVOURS, g_nonzeros

_POP = np.array([bin(i).count("1") for i in range(1 << 12)], dtype=np.int64)


def _times_generator(mu, md, coef, flavour: int, g: int):
    """(u monomials, d monomials, coefficients) times one generator on the
    right; monomials that already hold it vanish and are dropped."""
    bit = np.int64(1) << g
    own = mu if flavour == 0 else md
    keep = (own & bit) == 0
    above = _POP[own >> (g + 1)]
    sign = np.where(above & 1, -1, 1)
    coef = coef * sign
    own = own | bit
    if flavour == 0:
        mu = own
    else:
        md = own
    return mu[keep], md[keep], coef[keep]


def l_tensor(baryons: str, alpha, dirac_dim: int, G=None) -> dict:
    """{(U tuple, D tuple): L} with the zero entries dropped, for baryons like
    "PPNN" and one spin per baryon in the same order. ``G`` replaces the
    tensor of eq. def_g (optional; shape (D, 12, 12, 12), integer entries)."""
    if G is None:
        nz = g_nonzeros(dirac_dim)
    else:
        Ga = np.rint(np.asarray(G)).astype(np.int64)
        nz = {a: [((int(i), int(j), int(k)), int(Ga[a, i, j, k])) for i, j, k in zip(*np.nonzero(Ga[a]))]
              for a in range(Ga.shape[0])}
    mu = np.zeros(1, dtype=np.int64)
    md = np.zeros(1, dtype=np.int64)
    coef = np.ones(1, dtype=np.int64)
    for b, a in zip(baryons, alpha):
        fl = SLOT_FLAVOURS[b]
        parts_u, parts_d, parts_c = [], [], []
        for xi, gv in nz[int(a)]:
            u, d, c = mu, md, coef * int(round(gv))
            for slot in range(3):
                u, d, c = _times_generator(u, d, c, fl[slot], int(xi[slot]))
            parts_u.append(u)
            parts_d.append(d)
            parts_c.append(c)
        mu = np.concatenate(parts_u)
        md = np.concatenate(parts_d)
        coef = np.concatenate(parts_c)
        # collect equal monomials (exact integer sums)
        key = mu | (md << 12)
        order = np.argsort(key, kind="stable")
        key, coef = key[order], coef[order]
        if key.size == 0:
            return {}
        starts = np.flatnonzero(np.r_[True, key[1:] != key[:-1]])
        coef = np.add.reduceat(coef, starts)
        key = key[starts]
        live = coef != 0
        key, coef = key[live], coef[live]
        mu, md = key & 0xFFF, key >> 12
    out = {}
    for u, d, c in zip(mu.tolist(), md.tolist(), coef.tolist()):
        U = tuple(i for i in range(12) if u >> i & 1)
        D = tuple(i for i in range(12) if d >> i & 1)
        out[(U, D)] = int(c)
    return out

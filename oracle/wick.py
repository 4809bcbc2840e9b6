"""O1: the plain Wick definition of the correlator (oracle, test infrastructure).

Test infrastructure only (see ``oracle/__init__.py``).

Sec. 1 eq. C_baryons with the operators of Sec. 7 and the G tensors of
eq. def_g: every sink assignment xi' and source assignment xi of the 3A quark
slots, weighted by prod_k G(delta_k; xi'_k) prod_l G(alpha_l; xi_l), times the
Wick contraction of the quark fields. For each flavour q that contraction is
the signed sum over all permutations sigma of the q slots,

    sum_sigma sgn(sigma) prod_{i in q slots} S_q[xi'_i; xi_sigma(i)],

written out here permutation by permutation (no determinant routine), so the
work is n_u! n_d! times the number of (sink, source) assignment pairs: the
paper's naive operation count (Sec. 1). Global sign: + prod_q (the paper does
not fix it; it is the same for every component).
"""
from __future__ import annotations

import itertools

import numpy as np

from .gamma import SLOT_FLAVOURS, g_nonzeros, g_tensor_sources


def _perms_with_sign(n):
    out = []
    for p in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        out.append((p, -1.0 if inv % 2 else 1.0))
    return out


def _tuples(baryons, spins, dirac_dim, gnz=None):
    """All products of nonzero G entries (one per baryon): weights (n,) and the
    slot index tuples split by flavour: u (n, n_u), d (n, n_d). gnz: the
    nonzero entries {index: [((xi1, xi2, xi3), value), ...]} (default: those
    of G for dirac_dim)."""
    if gnz is None:
        gnz = g_nonzeros(dirac_dim)
    flav = [f for b in baryons for f in SLOT_FLAVOURS[b]]
    ws, us, ds = [], [], []
    for combo in itertools.product(*[gnz[int(s)] for s in spins]):
        w = 1.0
        idx = []
        for xi, g in combo:
            w *= g
            idx.extend(xi)
        ws.append(w)
        us.append([i for i, f in zip(idx, flav) if f == 0])
        ds.append([i for i, f in zip(idx, flav) if f == 1])
    return np.array(ws), np.array(us, dtype=np.int64), np.array(ds, dtype=np.int64)


def _flavour_contraction(S, rows, cols, chunk=1 << 16):
    """W[a, b] = sum_sigma sgn(sigma) prod_i S[rows[a, i], cols[b, sigma(i)]]."""
    n = rows.shape[1]
    W = np.zeros((rows.shape[0], cols.shape[0]), dtype=complex)
    if n == 0:
        W[:] = 1.0
        return W
    for perm, sgn in _perms_with_sign(n):
        term = np.ones_like(W)
        for i in range(n):
            term *= S[rows[:, i][:, None], cols[:, perm[i]][None, :]]
        W += sgn * term
    return W


def correlator(baryons: str, delta, alpha, dirac_dim: int, S_u, S_d) -> complex:
    """C(delta; alpha) at one site by explicit Wick enumeration (A <= 3)."""
    S_u = np.asarray(S_u, dtype=complex)
    S_d = np.asarray(S_d, dtype=complex)
    ws, us, ds = _tuples(baryons, delta, dirac_dim)
    wt, ut, dt = _tuples(baryons, alpha, dirac_dim)
    if len(ws) == 0 or len(wt) == 0:
        return 0j
    Wu = _flavour_contraction(S_u, us, ut)
    Wd = _flavour_contraction(S_d, ds, dt)
    return complex(ws @ (Wu * Wd) @ wt)


def correlator_sources(baryons: str, delta, chi, dirac_dim: int, S_list) -> complex:
    """C(delta; chi) at one site for N_s mutually orthogonal quark sources
    (Sec. 6), u = d, by explicit Wick enumeration (A <= 3).

    The sink is the single-source operator (G, eq. def_g); the source baryons
    carry chi = N_s * alpha + s and G~ (eq. G_tilde), whose quark indices are
    xi = N_s * kappa + s. A quark contracted from sink index xi' to source
    index xi propagates from source s: the matrix element is S_s[xi', kappa].
    S_list: (N_s, 12, 12) complex."""
    S_list = np.asarray(S_list, dtype=complex)
    ns = S_list.shape[0]
    nx = 3 * dirac_dim * ns
    # rectangular propagator: sink rows xi' (12), source columns xi (nx)
    S = np.zeros((12, nx), dtype=complex)
    for s in range(ns):
        for k in range(3 * dirac_dim):
            S[:, ns * k + s] = S_list[s, :, k]
    Gt = g_tensor_sources(dirac_dim, ns)
    src_nz = {}
    for c in range(Gt.shape[0]):
        nz = np.argwhere(Gt[c] != 0)
        src_nz[c] = [((int(i), int(j), int(k)), float(Gt[c, i, j, k])) for i, j, k in nz]
    ws, us, ds = _tuples(baryons, delta, dirac_dim)
    wt, ut, dt = _tuples(baryons, chi, dirac_dim, gnz=src_nz)
    if len(ws) == 0 or len(wt) == 0:
        return 0j
    Wu = _flavour_contraction(S, us, ut)
    Wd = _flavour_contraction(S, ds, dt)
    return complex(ws @ (Wu * Wd) @ wt)

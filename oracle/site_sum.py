"""Momentum-projected sum over sink sites (oracle, test infrastructure).

Test infrastructure only (see ``oracle/__init__.py``).

C(t, n) = sum_x exp(-2 pi i (n_x x / L_x + n_y y / L_y + n_z z / L_z)) C(x, t)
(Sec. 2: the sink function s(x) selects the momentum). Each product n_k x_k
is reduced modulo L_k in integers before the phase is formed, and every sum
is exactly rounded (``math.fsum`` on the real and imaginary parts).
"""
from __future__ import annotations

import math

import numpy as np


def phases(coords: np.ndarray, dims_xyz, mom) -> np.ndarray:
    """exp(-2 pi i n.x / L) for integer site coordinates (x, y, z)."""
    lx, ly, lz = dims_xyz
    n = np.asarray(mom, dtype=np.int64)
    r = [np.mod(n[0] * coords[:, 0], lx), np.mod(n[1] * coords[:, 1], ly), np.mod(n[2] * coords[:, 2], lz)]
    turns = r[0] / lx + r[1] / ly + r[2] / lz
    ang = -2.0 * np.pi * turns
    return np.cos(ang) + 1j * np.sin(ang)


def site_sum(C_sites: np.ndarray, coords: np.ndarray, dims_xyz, moms) -> np.ndarray:
    """C_sites: (n_sites, n_comp). Returns (n_mom, n_comp) complex128."""
    out = np.zeros((len(moms), C_sites.shape[1]), dtype=np.complex128)
    for q, mom in enumerate(moms):
        ph = phases(coords, dims_xyz, mom)
        prod = ph[:, None] * C_sites
        for c in range(C_sites.shape[1]):
            out[q, c] = complex(math.fsum(prod[:, c].real), math.fsum(prod[:, c].imag))
    return out


def scale_sum(scale_sites: np.ndarray) -> np.ndarray:
    """Error scale of a site sum: sum over sites of the per-site magnitude
    recursion (|phase| = 1). (n_sites, n_comp) -> (n_comp,)."""
    return np.array([math.fsum(scale_sites[:, c]) for c in range(scale_sites.shape[1])])

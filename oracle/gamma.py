"""Spin / colour conventions and the G^B tensors (oracle side).

Test infrastructure only (see ``oracle/__init__.py``).

Readings of the paper fixed here (the paper does not state them):

* combined spinor-colour index xi = 3 * spin + colour, 0-based (the paper only
  says the index runs over 12 values, Sec. 2);
* Euclidean Dirac representation (implied by Sec. 7, where P_nr keeps the
  upper two spinor components): gamma_k = [[0, -i sigma_k], [i sigma_k, 0]],
  gamma_4 = diag(1, 1, -1, -1), gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4;
* charge conjugation C = gamma_2 gamma_4;
* relativistic operators: Gamma_1 = 1, Gamma_2 = C gamma_5 (Sec. 1, Sec. 7);
  nonrelativistic: Gamma_1 = P_nr, Gamma_2 = C gamma_5 P_nr with
  P_nr = (1 + gamma_4) / 2 (Sec. 7);
* the same G^B tensor (eq. def_g) is used at the sink and at the source;
* baryon quark slots: proton (u, u, d), neutron (d, u, d) (Sec. 7).
"""
from __future__ import annotations

import itertools

import numpy as np

SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=complex),
    np.array([[0, -1j], [1j, 0]], dtype=complex),
    np.array([[1, 0], [0, -1]], dtype=complex),
]
Z2 = np.zeros((2, 2), dtype=complex)
I2 = np.eye(2, dtype=complex)


def gammas():
    """Euclidean Dirac-representation gamma_1..gamma_4 (list of 4x4)."""
    g = [np.block([[Z2, -1j * s], [1j * s, Z2]]) for s in SIGMA]
    g.append(np.block([[I2, Z2], [Z2, -I2]]))
    return g


def gamma5():
    g1, g2, g3, g4 = gammas()
    return g1 @ g2 @ g3 @ g4


def charge_conjugation():
    g = gammas()
    return g[1] @ g[3]


def p_nr():
    """Projector to the 'nonrelativistic' upper spinor components (Sec. 7)."""
    return 0.5 * (np.eye(4) + gammas()[3])


def gamma_pair(dirac_dim: int):
    """(Gamma_1, Gamma_2) for relativistic (dirac_dim=4) or nonrelativistic
    (dirac_dim=2) nucleon operators (Sec. 7)."""
    cg5 = charge_conjugation() @ gamma5()
    if dirac_dim == 4:
        return np.eye(4, dtype=complex), cg5
    if dirac_dim == 2:
        p = p_nr()
        return p.astype(complex), cg5 @ p
    raise ValueError("dirac_dim must be 2 or 4")


def epsilon():
    e = np.zeros((3, 3, 3))
    for p in itertools.permutations(range(3)):
        inv = sum(1 for i in range(3) for j in range(i + 1, 3) if p[i] > p[j])
        e[p] = -1.0 if inv % 2 else 1.0
    return e


def g_tensor(dirac_dim: int) -> np.ndarray:
    """Dense G(alpha; xi1, xi2, xi3) = (Gamma_1)_{alpha, s1} (Gamma_2)_{s2, s3}
    eps_{c1 c2 c3}, eq. def_g; shape (4, 12, 12, 12), real for these Gammas."""
    g1, g2 = gamma_pair(dirac_dim)
    eps = epsilon()
    G = np.zeros((4, 12, 12, 12), dtype=complex)
    for a in range(4):
        for x1, x2, x3 in itertools.product(range(12), repeat=3):
            s1, c1 = divmod(x1, 3)
            s2, c2 = divmod(x2, 3)
            s3, c3 = divmod(x3, 3)
            G[a, x1, x2, x3] = g1[a, s1] * g2[s2, s3] * eps[c1, c2, c3]
    assert np.allclose(G.imag, 0.0)
    return G.real.copy()


def g_nonzeros(dirac_dim: int):
    """{alpha: [((xi1, xi2, xi3), value), ...]} for the nonzero G entries."""
    G = g_tensor(dirac_dim)
    out = {}
    for a in range(4):
        nz = np.argwhere(G[a] != 0)
        out[a] = [((int(i), int(j), int(k)), float(G[a, i, j, k])) for i, j, k in nz]
    return out


# Flavour of each quark slot of a baryon (Sec. 7): 0 = u, 1 = d.
SLOT_FLAVOURS = {"P": (0, 0, 1), "N": (1, 0, 1)}


def g_tensor_sources(dirac_dim: int, n_sources: int) -> np.ndarray:
    """G~(chi; xi1, xi2, xi3) of Sec. 6 eq. G_tilde for n_sources mutually
    orthogonal quark sources: chi = n_sources * alpha + s and xi =
    n_sources * kappa + s (the combined spin-source index 2 alpha + s of
    Table 6 for two sources); G~ is G(alpha; kappa1, kappa2, kappa3) when all
    three quarks come from source s, else zero.
    Shape (dirac_dim * n_sources, 3 * dirac_dim * n_sources, ...)."""
    G = g_tensor(dirac_dim)
    nk = 3 * dirac_dim
    nc, nx = dirac_dim * n_sources, nk * n_sources
    out = np.zeros((nc, nx, nx, nx))
    for a in range(dirac_dim):
        for s in range(n_sources):
            chi = n_sources * a + s
            for k1, k2, k3 in zip(*np.nonzero(G[a, :nk, :nk, :nk])):
                out[chi, n_sources * k1 + s, n_sources * k2 + s, n_sources * k3 + s] = G[a, k1, k2, k3]
    return out

"""Seeded synthetic point-to-all quark propagators.

This module holds no contraction arithmetic: it only draws random numbers.
Both the CPU oracle and the CUDA path take their inputs from here, so the two
sides see identical propagators without sharing any of the method's code.

Recipe (the paper uses no gauge ensemble, so these stand in for real
propagators):

* one (configuration, time slice) pair is a "slab" of Lz*Ly*Lx sink sites;
* every slab has its own generator, ``numpy.random.default_rng(
  SeedSequence([seed, cfg, t]))``, so any slab can be regenerated alone;
* it draws ``standard_normal((Lz, Ly, Lx, 12, 12, 2))``; entry
  ``S[z, y, x, row, col] = (g[..., 0] + 1j * g[..., 1]) * exp(-lam * t)``;
* ``row`` is the sink spinor-colour index, ``col`` the source index, both
  packed as ``3 * spin + colour``;
* u and d quarks share one field (u = d);
* with N_s quark sources (Sec. 6) a site holds N_s such matrices, axis
  ``[..., s, row, col]``; source 0 is the single-source slab above and source
  s >= 1 draws the same shape from its own stream ``SeedSequence([seed, cfg,
  t, s])``;
* complex64 storage is the complex128 value rounded to nearest; every consumer
  (oracle included) promotes the rounded values, so storage rounding is never
  counted as a compute error;
* ``eps`` (optional) turns the same draws into near-identity propagators,
  ``S = (1 + eps * (g0 + i g1)) * exp(-lam * t)``: random Gaussian matrices
  make the correlator cancel by many orders of magnitude against the sum of
  the magnitudes of its terms (8Be: 1e-13), while near the identity the two
  are of one order, so an error bound relative to that sum can tell a right
  result from a wrong one.
"""
from __future__ import annotations

import numpy as np

__all__ = ["slab", "slab_sources", "field", "site_coords"]


def _shape(g, eps):
    z = g[..., 0] + 1j * g[..., 1]
    if eps is None:
        return z
    return np.eye(12) + float(eps) * z


def slab(seed: int, cfg: int, t: int, dims, lam: float, dtype=np.complex128, eps=None) -> np.ndarray:
    """Propagators of one (cfg, t) slab, shape (Lz, Ly, Lx, 12, 12)."""
    lz, ly, lx = (int(d) for d in dims)
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), int(cfg), int(t)]))
    g = rng.standard_normal((lz, ly, lx, 12, 12, 2))
    s = _shape(g, eps) * np.exp(-float(lam) * float(t))
    return s.astype(dtype)


def slab_sources(seed: int, cfg: int, t: int, dims, lam: float, n_src: int,
                 dtype=np.complex128, eps=None) -> np.ndarray:
    """Propagators of N_s sources for one slab, shape (Lz, Ly, Lx, n_src, 12, 12)."""
    lz, ly, lx = (int(d) for d in dims)
    out = np.empty((lz, ly, lx, int(n_src), 12, 12), dtype=dtype)
    out[..., 0, :, :] = slab(seed, cfg, t, dims, lam, dtype, eps)
    for s in range(1, int(n_src)):
        rng = np.random.default_rng(np.random.SeedSequence([int(seed), int(cfg), int(t), s]))
        g = rng.standard_normal((lz, ly, lx, 12, 12, 2))
        out[..., s, :, :] = (_shape(g, eps) * np.exp(-float(lam) * float(t))).astype(dtype)
    return out


def field(seed: int, n_cfg: int, nt: int, dims, lam: float, dtype=np.complex128,
          cfgs=None, ts=None, n_src: int = 0, eps=None) -> np.ndarray:
    """Stack of slabs, shape (n_cfg', nt', Lz, Ly, Lx, 12, 12), or
    (n_cfg', nt', Lz, Ly, Lx, n_src, 12, 12) when n_src >= 1.

    ``cfgs`` / ``ts`` select a subset of configurations / time slices (default:
    all); each slab is generated from its own (seed, cfg, t) stream. ``eps``
    gives near-identity propagators from the same draws (module docstring).
    """
    cfgs = list(range(n_cfg)) if cfgs is None else list(cfgs)
    ts = list(range(nt)) if ts is None else list(ts)
    lz, ly, lx = (int(d) for d in dims)
    site = (12, 12) if n_src < 1 else (int(n_src), 12, 12)
    out = np.empty((len(cfgs), len(ts), lz, ly, lx) + site, dtype=dtype)
    for i, c in enumerate(cfgs):
        for j, t in enumerate(ts):
            out[i, j] = (slab(seed, c, t, dims, lam, dtype, eps) if n_src < 1
                         else slab_sources(seed, c, t, dims, lam, n_src, dtype, eps))
    return out


def site_coords(dims) -> np.ndarray:
    """(x, y, z) integer coordinates of the sites of a slab in storage order
    (z slowest, x fastest), shape (Lz*Ly*Lx, 3)."""
    lz, ly, lx = (int(d) for d in dims)
    z, y, x = np.meshgrid(np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)

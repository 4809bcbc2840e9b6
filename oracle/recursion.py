"""O3 driver: compiles ``recursion.c`` with gcc and calls it through ctypes.

Test infrastructure only (see ``oracle/__init__.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from .gamma import g_tensor
from .minors import nucleus_components

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "recursion.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_o3.so")
# the same source with 64-bit keys: 24 quark index values, 8 source baryon
# index values (two relativistic quark sources, Sec. 6)
_LIB_WIDE = os.path.join(_OUT_DIR, "liboracle_o3w.so")
_lock = threading.Lock()
_libs = {}


def build(force: bool = False) -> str:
    """Compile the O3 oracle libraries (gcc, OpenMP): the 32-bit-key one and
    the wide one (-DO3_WIDE); returns the path of the first."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    for lib, extra in ((_LIB, []), (_LIB_WIDE, ["-DO3_WIDE"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
            tmp = lib + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", *extra, "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, lib)
    return _LIB


def _load(wide: bool = False):
    with _lock:
        if wide not in _libs:
            build()
            lib = ctypes.CDLL(_LIB_WIDE if wide else _LIB)
            P = ctypes.c_void_p
            lib.o3_plan_build.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int, P, P,
                                          ctypes.POINTER(ctypes.c_void_p)]
            lib.o3_plan_build.restype = ctypes.c_int
            lib.o3_free.argtypes = [P]
            lib.o3_n_ops.argtypes = [P, P, P]
            lib.o3_n_ops.restype = ctypes.c_int64
            lib.o3_req_nl.argtypes = [P, ctypes.c_int]
            lib.o3_req_nl.restype = ctypes.c_int64
            lib.o3_norm.argtypes = [P]
            lib.o3_norm.restype = ctypes.c_double
            lib.o3_eval.argtypes = [P, ctypes.c_int64, P, P, P, ctypes.c_int]
            lib.o3_eval.restype = ctypes.c_int
            lib.o3_blocks.argtypes = [P, ctypes.c_int64, P, P, P, P, P]
            lib.o3_blocks.restype = ctypes.c_int
            lib.o3_eval_blocks.argtypes = [P, ctypes.c_int64, P, P, P, P, P, P]
            lib.o3_eval_blocks.restype = ctypes.c_int
            lib.o3_stage_keys.argtypes = [P, ctypes.c_int, P]
            lib.o3_stage_keys.restype = ctypes.c_int64
            lib.o3_plan_set_sink.argtypes = [P, P]
            lib.o3_plan_set_sink.restype = None
            _libs[wide] = lib
    return _libs[wide]


def paper_path(n_p: int, n_n: int) -> list:
    """Recursion order of Sec. 7: all baryons of the more numerous species
    first; on a tie, neutrons first. 0 = proton, 1 = neutron."""
    if n_p > n_n:
        return [0] * n_p + [1] * n_n
    return [1] * n_n + [0] * n_p


def _padded(G, nsp=4, nq=12) -> np.ndarray:
    Gd = np.asarray(G)
    Gp = np.zeros((nsp, nq, nq, nq))
    Gp[: Gd.shape[0], : Gd.shape[1], : Gd.shape[2], : Gd.shape[3]] = Gd
    return np.ascontiguousarray(np.rint(Gp).astype(np.int8))


def source_columns(S, dirac_dim: int) -> np.ndarray:
    """Propagators of N_s sources, (..., N_s, 12, 12), as one matrix per site
    with source quark index xi = N_s * kappa + s (Sec. 6): column xi is column
    kappa of source s, for kappa < 3 * dirac_dim (the index values G~ uses).
    Returns (..., 12, 12) complex128, or (..., 12, 24) when 3 dirac_dim N_s
    exceeds 12; columns beyond 3 dirac_dim N_s are zero."""
    S = np.asarray(S, dtype=np.complex128)
    ns = S.shape[-3]
    nk = 3 * dirac_dim
    if nk * ns > 24:
        raise ValueError("3 * dirac_dim * n_sources must not exceed 24")
    out = np.zeros(S.shape[:-3] + (12, 12 if nk * ns <= 12 else 24), dtype=np.complex128)
    for s in range(ns):
        for k in range(nk):
            out[..., :, ns * k + s] = S[..., s, :, k]
    return out


class Plan:
    """Symbolic part of O3 for one nucleus and a list of (sink, source) spin
    assignments (protons first, each species sorted ascending)."""

    def __init__(self, n_p: int, n_n: int, dirac_dim: int, requests=None, path=None, G=None, G_sink=None,
                 wide=None):
        Gsrc = g_tensor(dirac_dim) if G is None else np.asarray(G)
        # the 64-bit-key build takes more than 12 quark or 4 source baryon
        # index values (two relativistic quark sources)
        self.wide = bool(wide) if wide is not None else (Gsrc.shape[0] > 4 or Gsrc.shape[1] > 12)
        self.nq = 24 if self.wide else 12
        lib = _load(self.wide)
        self.n_p, self.n_n, self.dim = n_p, n_n, dirac_dim
        self.A = n_p + n_n
        if requests is None:
            comps = nucleus_components(n_p, n_n, dirac_dim)
            requests = [(d, a) for d in comps for a in comps]
        self.requests = [(tuple(d), tuple(a)) for d, a in requests]
        self.path = list(paper_path(n_p, n_n) if path is None else path)
        # G: optional replacement tensor (e.g. the two-source G~ of Sec. 6),
        # at most (4, 12, 12, 12), or (8, 24, 24, 24) for a wide plan,
        # zero-padded to that shape; G_sink: the tensor of the blocks when it
        # differs (one sink, several sources), at most (4, 12, 12, 12)
        G = _padded(Gsrc, 8 if self.wide else 4, self.nq)
        snk = np.ascontiguousarray(np.array([d for d, _ in self.requests], dtype=np.int8).reshape(-1))
        src = np.ascontiguousarray(np.array([a for _, a in self.requests], dtype=np.int8).reshape(-1))
        pa = np.ascontiguousarray(np.array(self.path, dtype=np.int8))
        h = ctypes.c_void_p()
        rc = lib.o3_plan_build(n_p, n_n, dirac_dim, pa.ctypes.data, G.ctypes.data, len(self.requests),
                               snk.ctypes.data if snk.size else None, src.ctypes.data if src.size else None,
                               ctypes.byref(h))
        if rc != 0:
            raise ValueError("invalid nucleus / request for O3")
        self._h = h
        self._lib = lib
        if G_sink is not None or self.wide:
            self._gs = _padded(g_tensor(dirac_dim) if G_sink is None else G_sink)
            lib.o3_plan_set_sink(h, self._gs.ctypes.data)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.o3_free(h)
            self._h = None

    def ops(self):
        """(N_Lambda, ops per step, needed keys per stage)."""
        per = np.zeros(16, dtype=np.int64)
        st = np.zeros(16, dtype=np.int64)
        t = self._lib.o3_n_ops(self._h, per.ctypes.data, st.ctypes.data)
        return int(t), per[: self.A - 1].tolist(), st[: self.A].tolist()

    def stage_keys(self, m: int) -> np.ndarray:
        """Needed components of stage m (1-based) after the backward pruning,
        as packed keys (proton spins | neutron spins << 4 | u set << 8 |
        d set << 20; wide plans: spins | spins << 8 | u << 16 | d << 40),
        ascending."""
        n = int(self._lib.o3_stage_keys(self._h, m, None))
        out = np.zeros(max(n, 1), dtype=np.uint64 if self.wide else np.uint32)
        self._lib.o3_stage_keys(self._h, m, out.ctypes.data)
        return out[:n]

    def n_l(self):
        """Nonzero L entries per request."""
        return [int(self._lib.o3_req_nl(self._h, r)) for r in range(len(self.requests))]

    @property
    def norm(self) -> float:
        return float(self._lib.o3_norm(self._h))

    def evaluate(self, S: np.ndarray, batch: int = 16):
        """Per-site correlators. S: (..., 12, 12) complex, u = d (wide plans:
        (..., 12, 24), sink rows x source columns; 12 columns are padded).
        Returns (C, scale): C (n_sites, n_req) complex128, scale the
        magnitude recursion "sum |terms|" (n_sites, n_req)."""
        S = self._tiles(S)
        n = S.shape[0]
        out = np.zeros((n, len(self.requests)), dtype=np.complex128)
        sc = np.zeros((n, len(self.requests)), dtype=np.float64)
        rc = self._lib.o3_eval(self._h, n, S.ctypes.data, out.ctypes.data, sc.ctypes.data, int(batch))
        if rc != 0:
            raise RuntimeError("o3_eval failed")
        return out, sc

    def _tiles(self, S):
        S = np.asarray(S, dtype=np.complex128)
        S = S.reshape((-1, 12, S.shape[-1]))
        if S.shape[-1] < self.nq:
            S = np.concatenate([S, np.zeros(S.shape[:-1] + (self.nq - S.shape[-1],), dtype=S.dtype)], axis=-1)
        return np.ascontiguousarray(S)

    def blocks(self, S: np.ndarray):
        """Antisymmetric block components per site (Sec. 2, Sec. 4):
        (f_P, f_N, |f_P|, |f_N|), each (n_sites, 4, nq, nq, nq)."""
        S = self._tiles(S)
        n = S.shape[0]
        q = self.nq
        shp = (n, 4, q, q, q)
        fp = np.zeros(shp, dtype=np.complex128)
        fn = np.zeros(shp, dtype=np.complex128)
        mp = np.zeros(shp)
        mn = np.zeros(shp)
        self._lib.o3_blocks(self._h, n, S.ctypes.data, fp.ctypes.data, fn.ctypes.data, mp.ctypes.data, mn.ctypes.data)
        return fp, fn, mp, mn

    def evaluate_blocks(self, fp, fn, mp, mn):
        """Recursion and contraction from given blocks (e.g. momentum-projected
        ones): arrays (n_items, 4, nq, nq, nq) as from ``blocks``. Returns
        (C, scale), each (n_items, n_req)."""
        arrs = [np.ascontiguousarray(np.asarray(a, dtype=t)) for a, t in
                ((fp, np.complex128), (fn, np.complex128), (mp, np.float64), (mn, np.float64))]
        n = arrs[0].shape[0]
        out = np.zeros((n, len(self.requests)), dtype=np.complex128)
        sc = np.zeros((n, len(self.requests)), dtype=np.float64)
        self._lib.o3_eval_blocks(self._h, n, *[a.ctypes.data for a in arrs], out.ctypes.data, sc.ctypes.data)
        return out, sc

"""Python binding of libmbc (recursive multibaryon correlation functions).

Argument marshalling only: every step of the contraction runs in the CUDA
library (``csrc/``), the term lists are built by its host C++ builder. The
names follow the C ABI in ``include/mbc.h`` without the ``mbc_`` prefix.
Loading fails loudly when the compiled library is missing: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "MbcError", "load", "build_term_list", "TermList", "contract", "sync_status", "release_scratch",
    "FP64", "MIXED", "C128", "C64", "PROTON", "NEUTRON", "timing_enable", "timing_read", "fma_probe",
    "contract_noalloc", "check_wait_timeout",
]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmbc.so")

FP64, MIXED = 0, 1
C128, C64 = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
PROTON, NEUTRON = 0, 1
SPIN_ALL, SPIN_LISTED, SPIN_PROJECTED = 0, 1, 2
MAX_A = 16
MAX_MOM = 32

STATUS = {0: "MBC_OK", 1: "MBC_ERR_INVALID_ARG", 2: "MBC_ERR_PAULI_FORBIDDEN", 3: "MBC_ERR_OOM",
          4: "MBC_ERR_CUDA", 5: "MBC_ERR_TIMEOUT", 6: "MBC_ERR_UNSUPPORTED"}


class MbcError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}")


class OpSpec(ctypes.Structure):
    _fields_ = [("n_p", ctypes.c_int32), ("n_n", ctypes.c_int32), ("dirac_dim", ctypes.c_int32),
                ("n_sources", ctypes.c_int32), ("spin_mode", ctypes.c_int32), ("n_spin_sel", ctypes.c_int32),
                ("snk_spins", ctypes.c_void_p), ("src_spins", ctypes.c_void_p), ("path_len", ctypes.c_int32),
                ("path", ctypes.c_void_p), ("n_proj", ctypes.c_int32), ("term_proj", ctypes.c_void_p),
                ("term_coef", ctypes.c_void_p), ("n_sinks", ctypes.c_int32), ("list_free", ctypes.c_int32)]


class ListStats(ctypes.Structure):
    _fields_ = [("A", ctypes.c_int32), ("n_steps", ctypes.c_int32), ("path", ctypes.c_int8 * MAX_A),
                ("n_ops_total", ctypes.c_int64), ("n_ops", ctypes.c_int64 * MAX_A),
                ("ops_per_z", ctypes.c_int64 * MAX_A), ("stage_size", ctypes.c_int64 * MAX_A),
                ("stage_bound", ctypes.c_int64 * MAX_A), ("q_bound", ctypes.c_int64 * MAX_A),
                ("block_size", ctypes.c_int64), ("n_comp", ctypes.c_int32), ("n_l_total", ctypes.c_int64),
                ("norm", ctypes.c_double), ("n_parts", ctypes.c_int32), ("dense_mask", ctypes.c_uint32),
                ("op_bytes", ctypes.c_int64)]


class ListPart(ctypes.Structure):
    _fields_ = [("n_p", ctypes.c_int32), ("n_n", ctypes.c_int32), ("c0", ctypes.c_int32), ("c1", ctypes.c_int32)]


class Props(ctypes.Structure):
    _fields_ = [("s_u", ctypes.c_void_p), ("s_d", ctypes.c_void_p), ("dtype", ctypes.c_int32),
                ("memory", ctypes.c_int32), ("n_cfg", ctypes.c_int32), ("nt", ctypes.c_int32),
                ("lx", ctypes.c_int32), ("ly", ctypes.c_int32), ("lz", ctypes.c_int32),
                ("stride_cfg", ctypes.c_int64), ("stride_t", ctypes.c_int64), ("n_src", ctypes.c_int32)]


class Tune(ctypes.Structure):
    _fields_ = [("sites_per_cta", ctypes.c_int32), ("threads_per_cta", ctypes.c_int32),
                ("wave_sites", ctypes.c_int32), ("regime", ctypes.c_int32), ("zchunk", ctypes.c_int32),
                ("wave_order", ctypes.c_int32), ("list_free", ctypes.c_int32)]

    FIELDS = ("sites_per_cta", "threads_per_cta", "wave_sites", "regime", "zchunk", "wave_order", "list_free")


class ContractOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("n_mom", ctypes.c_int32), ("mom", ctypes.c_void_p),
                ("t0", ctypes.c_int32), ("t1", ctypes.c_int32), ("tune", ctypes.c_void_p),
                ("sink_mode", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load libmbc.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or os.environ.get("MBC_LIB") or LIB_PATH
        if not os.path.exists(p):
            raise OSError(f"libmbc.so not found at {p}: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(p)
        V = ctypes.c_void_p
        lib.mbc_status_string.argtypes = [ctypes.c_int]
        lib.mbc_status_string.restype = ctypes.c_char_p
        lib.mbc_build_term_list.argtypes = [ctypes.POINTER(OpSpec), ctypes.POINTER(V)]
        lib.mbc_build_term_list.restype = ctypes.c_int
        lib.mbc_save_term_list.argtypes = [V, ctypes.c_char_p]
        lib.mbc_save_term_list.restype = ctypes.c_int
        lib.mbc_load_term_list.argtypes = [ctypes.c_char_p, ctypes.POINTER(V)]
        lib.mbc_load_term_list.restype = ctypes.c_int
        lib.mbc_build_combined.argtypes = [ctypes.POINTER(OpSpec), ctypes.c_int32, ctypes.POINTER(V)]
        lib.mbc_build_combined.restype = ctypes.c_int
        lib.mbc_term_list_part.argtypes = [V, ctypes.c_int32, ctypes.POINTER(ListPart)]
        lib.mbc_term_list_part.restype = ctypes.c_int
        lib.mbc_term_list_stats.argtypes = [V, ctypes.POINTER(ListStats)]
        lib.mbc_term_list_stats.restype = ctypes.c_int
        lib.mbc_term_list_components.argtypes = [V, V, V]
        lib.mbc_term_list_components.restype = ctypes.c_int
        lib.mbc_term_list_n_l.argtypes = [V, ctypes.c_int32]
        lib.mbc_term_list_n_l.restype = ctypes.c_int64
        lib.mbc_free_term_list.argtypes = [V]
        lib.mbc_free_term_list.restype = None
        lib.mbc_contract.argtypes = [ctypes.POINTER(Props), ctypes.POINTER(V), ctypes.c_int32,
                                     ctypes.POINTER(ContractOpts), V, V]
        lib.mbc_contract.restype = ctypes.c_int
        lib.mbc_contract_noalloc.argtypes = [ctypes.POINTER(Props), V, ctypes.POINTER(ContractOpts), V, V]
        lib.mbc_contract_noalloc.restype = ctypes.c_int
        lib.mbc_sync_status.argtypes = [V]
        lib.mbc_sync_status.restype = ctypes.c_int
        lib.mbc_check_wait_timeout.argtypes = [ctypes.c_uint32, V]
        lib.mbc_check_wait_timeout.restype = ctypes.c_int
        lib.mbc_release_scratch.argtypes = []
        lib.mbc_release_scratch.restype = None
        lib.mbc_timing_enable.argtypes = [ctypes.c_int32]
        lib.mbc_timing_enable.restype = None
        lib.mbc_timing_read.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        lib.mbc_timing_read.restype = ctypes.c_int
        lib.mbc_fma_probe.argtypes = [ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
        lib.mbc_fma_probe.restype = ctypes.c_int
        lib.mbc_kernel_launches.argtypes = []
        lib.mbc_kernel_launches.restype = ctypes.c_int64
        lib.mbc_version.argtypes = []
        lib.mbc_version.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _check(rc: int, what: str, ok=(0,)):
    if rc not in ok:
        raise MbcError(rc, what)
    return rc


class TermList:
    """Owning handle of an ``mbc_term_list``."""

    def __init__(self, handle, status: int, spec: dict):
        self._h = handle
        self.status = status
        self.spec = spec
        self._lib = load()

    @property
    def handle(self):
        return self._h

    @property
    def pauli_forbidden(self) -> bool:
        return self.status == 2

    def stats(self) -> dict:
        """``mbc_term_list_stats`` as a dict (a list never changes: read once)."""
        if getattr(self, "_stats", None) is None:
            self._stats = self._read_stats()
        return {k: list(v) if isinstance(v, list) else v for k, v in self._stats.items()}

    def _read_stats(self) -> dict:
        st = ListStats()
        _check(self._lib.mbc_term_list_stats(self._h, ctypes.byref(st)), "mbc_term_list_stats")
        A = st.A
        return {
            "A": A, "n_steps": st.n_steps, "path": list(st.path[:A]), "n_ops_total": st.n_ops_total,
            "n_ops": list(st.n_ops[: st.n_steps]), "ops_per_z": list(st.ops_per_z[: st.n_steps]),
            "stage_size": list(st.stage_size[:A]), "stage_bound": list(st.stage_bound[:A]),
            "q_bound": list(st.q_bound[: st.n_steps]), "block_size": st.block_size, "n_comp": st.n_comp,
            "n_l_total": st.n_l_total, "norm": st.norm, "n_parts": st.n_parts,
            "dense_steps": [m + 1 for m in range(st.n_steps) if st.dense_mask >> m & 1], "op_bytes": st.op_bytes,
        }

    def parts(self):
        """Nuclei of the list: [{"n_p", "n_n", "c0", "c1"}], outputs [c0, c1) each."""
        out = []
        for j in range(self.stats()["n_parts"]):
            p = ListPart()
            _check(self._lib.mbc_term_list_part(self._h, j, ctypes.byref(p)), "mbc_term_list_part")
            out.append({"n_p": p.n_p, "n_n": p.n_n, "c0": p.c0, "c1": p.c1})
        return out

    def components(self):
        st = self.stats()
        n, A = st["n_comp"], st["A"]
        snk = np.zeros(max(n * A, 1), dtype=np.int8)
        src = np.zeros(max(n * A, 1), dtype=np.int8)
        if n:
            _check(self._lib.mbc_term_list_components(self._h, snk.ctypes.data, src.ctypes.data),
                   "mbc_term_list_components")
        return [(tuple(snk[i * A:(i + 1) * A].tolist()), tuple(src[i * A:(i + 1) * A].tolist())) for i in range(n)]

    def save(self, path: str):
        """``mbc_save_term_list``: write the list to a file."""
        _check(self._lib.mbc_save_term_list(self._h, os.fsencode(path)), "mbc_save_term_list")

    def n_l(self, c: int) -> int:
        return int(self._lib.mbc_term_list_n_l(self._h, c))

    def free(self):
        if self._h:
            self._lib.mbc_free_term_list(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _op_spec(n_p, n_n, dirac_dim, spins, path, n_sources, projections, n_sinks, keep, list_free=False):
    """Fill an OpSpec; arrays it points to are appended to keep."""
    A = n_p + n_n
    spec = OpSpec()
    spec.n_p, spec.n_n, spec.dirac_dim, spec.n_sources = n_p, n_n, dirac_dim, n_sources
    spec.n_sinks = n_sinks
    spec.list_free = 1 if list_free else 0
    if projections is not None:
        if spins is not None:
            raise ValueError("give spins or projections, not both")
        terms = [(p, s, a, w) for p, proj in enumerate(projections) for (s, a, w) in proj]
        snk = np.ascontiguousarray(np.array([t[1] for t in terms], dtype=np.int8).reshape(-1))
        src = np.ascontiguousarray(np.array([t[2] for t in terms], dtype=np.int8).reshape(-1))
        tp = np.ascontiguousarray(np.array([t[0] for t in terms], dtype=np.int32))
        tw = np.ascontiguousarray(np.array([t[3] for t in terms], dtype=np.float64))
        if snk.size != len(terms) * A or src.size != len(terms) * A:
            raise ValueError("each spin assignment needs A entries")
        spec.spin_mode = SPIN_PROJECTED
        spec.n_spin_sel, spec.n_proj = len(terms), len(projections)
        spec.snk_spins, spec.src_spins = snk.ctypes.data, src.ctypes.data
        spec.term_proj, spec.term_coef = tp.ctypes.data, tw.ctypes.data
        keep += [snk, src, tp, tw]
    elif spins is None:
        spec.spin_mode = SPIN_ALL
    else:
        spec.spin_mode = SPIN_LISTED
        snk = np.ascontiguousarray(np.array([s for s, _ in spins], dtype=np.int8).reshape(-1))
        src = np.ascontiguousarray(np.array([a for _, a in spins], dtype=np.int8).reshape(-1))
        if snk.size != len(spins) * A or src.size != len(spins) * A:
            raise ValueError("each spin assignment needs A entries")
        spec.n_spin_sel = len(spins)
        spec.snk_spins, spec.src_spins = snk.ctypes.data, src.ctypes.data
        keep += [snk, src]
    if path is not None:
        pa = np.ascontiguousarray(np.array(path, dtype=np.int8))
        spec.path_len, spec.path = len(path), pa.ctypes.data
        keep.append(pa)
    return spec


def load_term_list(path: str, spec=None) -> TermList:
    """``mbc_load_term_list``: a list written by ``TermList.save``."""
    lib = load()
    h = ctypes.c_void_p()
    rc = lib.mbc_load_term_list(os.fsencode(path), ctypes.byref(h))
    _check(rc, "mbc_load_term_list", ok=(0, 2))
    return TermList(h, rc, spec or {"file": path})


def _cache_path(cache_dir: str, spec: dict) -> str:
    import hashlib
    key = repr(sorted(spec.items())) + load().mbc_version().decode()
    return os.path.join(cache_dir, "mbc_list_" + hashlib.sha256(key.encode()).hexdigest()[:24] + ".bin")


def build_term_list(n_p: int, n_n: int, dirac_dim: int = 4, spins=None, path=None, n_sources: int = 1,
                    projections=None, n_sinks: int = 1, list_free: bool = False, cache_dir=None) -> TermList:
    """``mbc_build_term_list``. spins: None for every independent component,
    or a list of (sink spins, source spins) pairs, protons first.
    projections: instead of spins, a list of projections, each a list of
    (sink spins, source spins, real weight) terms (Sec. 5); one output each.
    list_free: store no operation arrays (splits regenerated on the GPU).
    cache_dir: a directory of saved lists keyed by a hash of these
    arguments; the list is loaded from there when present, else built and
    saved there."""
    spec_d = {"n_p": n_p, "n_n": n_n, "dirac_dim": dirac_dim, "spins": spins, "path": path,
              "projections": projections, "n_sources": n_sources, "n_sinks": n_sinks, "list_free": list_free}
    if cache_dir is not None:
        fn = _cache_path(cache_dir, spec_d)
        if os.path.exists(fn):
            try:
                return load_term_list(fn, spec_d)
            except MbcError:
                pass  # unreadable or from another build: rebuild and overwrite
        tl = build_term_list(n_p, n_n, dirac_dim, spins, path, n_sources, projections, n_sinks, list_free)
        os.makedirs(cache_dir, exist_ok=True)
        tmp = f"{fn}.{os.getpid()}.tmp"
        tl.save(tmp)
        os.replace(tmp, fn)
        return tl
    lib = load()
    keep = []
    spec = _op_spec(n_p, n_n, dirac_dim, spins, path, n_sources, projections, n_sinks, keep, list_free)
    h = ctypes.c_void_p()
    rc = lib.mbc_build_term_list(ctypes.byref(spec), ctypes.byref(h))
    _check(rc, "mbc_build_term_list", ok=(0, 2))
    return TermList(h, rc, {"n_p": n_p, "n_n": n_n, "dirac_dim": dirac_dim, "spins": spins, "path": path,
                            "projections": projections, "n_sources": n_sources, "n_sinks": n_sinks,
                            "list_free": list_free})


def build_combined(nuclei, dirac_dim: int = 4, path=None, n_sources: int = 1, n_sinks: int = 1) -> TermList:
    """``mbc_build_combined``: one list for several nuclei on one recursion
    path (Sec. 7). nuclei: list of dicts with "n_p", "n_n" and optionally
    "spins" or "projections" (as for build_term_list); path: the order of the
    largest nucleus (None: the paper's rule). Outputs follow the nuclei in
    the order given (``TermList.parts``)."""
    lib = load()
    if not nuclei:
        raise ValueError("no nuclei given")
    keep = []
    big = max(range(len(nuclei)), key=lambda j: nuclei[j]["n_p"] + nuclei[j]["n_n"])
    arr = (OpSpec * len(nuclei))()
    for j, nu in enumerate(nuclei):
        arr[j] = _op_spec(nu["n_p"], nu["n_n"], dirac_dim, nu.get("spins"), path if j == big else None, n_sources,
                          nu.get("projections"), n_sinks, keep)
    h = ctypes.c_void_p()
    rc = lib.mbc_build_combined(arr, len(nuclei), ctypes.byref(h))
    _check(rc, "mbc_build_combined")
    return TermList(h, rc, {"nuclei": nuclei, "dirac_dim": dirac_dim, "path": path, "n_sources": n_sources,
                            "n_sinks": n_sinks})


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


SINK_POINT, SINK_BLOCK_MOMENTUM = 0, 1


def contract(field, lists, precision: int = FP64, moms=((0, 0, 0),), t0: int = 0, t1: int = 0, tune=None,
             out=None, stream=None, dims=None, sink: int = SINK_POINT):
    """``mbc_contract`` on a u = d propagator field.

    field: torch tensor (device memory) or numpy array (host memory) of shape
    (n_cfg, nt, Lz, Ly, Lx, 12, 12), or (n_cfg, nt, Lz, Ly, Lx, n_src, 12, 12)
    for lists built with n_sources = n_src (Sec. 6), complex128 or complex64,
    contiguous. Returns out: complex128 (n_cfg, n_lists, t1 - t0, n_mom / n_sinks,
    n_comp_max) on the same side as the field; lists with n_sinks > 1 need
    sink=SINK_BLOCK_MOMENTUM and take the momenta in groups of n_sinks.
    """
    lib = load()
    lists = list(lists)
    is_np = isinstance(field, np.ndarray)
    if is_np:
        if field.dtype not in (np.complex128, np.complex64) or not field.flags.c_contiguous:
            raise ValueError("field must be a C-contiguous complex128/complex64 array")
        dtype = C128 if field.dtype == np.complex128 else C64
        ptr = field.ctypes.data
        shape = field.shape
    else:
        import torch
        if field.dtype not in (torch.complex128, torch.complex64) or not field.is_contiguous():
            raise ValueError("field must be a contiguous complex128/complex64 tensor")
        dtype = C128 if field.dtype == torch.complex128 else C64
        ptr = field.data_ptr()
        shape = tuple(field.shape)
    if len(shape) not in (7, 8) or shape[-2:] != (12, 12):
        raise ValueError("field shape must be (n_cfg, nt, Lz, Ly, Lx, [n_src,] 12, 12)")
    n_cfg, nt, lz, ly, lx = shape[:5]
    n_src = shape[5] if len(shape) == 8 else 1
    t1e = nt if t1 == 0 else t1
    moms = np.ascontiguousarray(np.array(moms, dtype=np.int32).reshape(-1, 3))
    comp_max = max(1, max(tl.stats()["n_comp"] for tl in lists))
    n_k = max(1, int(lists[0].spec.get("n_sinks", 1) or 1)) if lists else 1
    oshape = (n_cfg, len(lists), t1e - t0, moms.shape[0] // n_k, comp_max)
    if out is None:
        if is_np:
            out = np.zeros(oshape, dtype=np.complex128)
        else:
            import torch
            out = torch.empty(oshape, dtype=torch.complex128, device=field.device)  # the library zero-fills
    optr = out.ctypes.data if is_np else out.data_ptr()
    pr = Props(ptr, ptr, dtype, MEM_HOST if is_np else MEM_DEVICE, n_cfg, nt, lx, ly, lz, 0, 0, n_src)
    tn = None
    if tune is not None:
        unknown = set(tune) - set(Tune.FIELDS)
        if unknown:
            raise ValueError(f"unknown tune fields {sorted(unknown)}")
        tn = Tune(*[int(tune.get(f, 0)) for f in Tune.FIELDS])
    op = ContractOpts(precision, moms.shape[0], moms.ctypes.data, t0, t1, ctypes.addressof(tn) if tn else None, sink)
    handles = (ctypes.c_void_p * len(lists))(*[tl.handle for tl in lists])
    rc = lib.mbc_contract(ctypes.byref(pr), handles, len(lists), ctypes.byref(op), optr, _stream_ptr(stream))
    _check(rc, "mbc_contract")
    return out


def contract_noalloc(field, term_list, out, moms=((0, 0, 0),), t0: int = 0, t1: int = 0, stream=None):
    """``mbc_contract_noalloc``: FP64 contraction of one list into a
    caller-allocated device tensor, with no device allocation inside the
    library (its scratch is a static 8 MiB device array). The list must have
    been used once with ``contract`` on this device. Returns ``out``."""
    lib = load()
    import torch
    if field.dtype not in (torch.complex128, torch.complex64) or not field.is_contiguous():
        raise ValueError("field must be a contiguous complex128/complex64 tensor")
    if out.dtype != torch.complex128 or not out.is_contiguous():
        raise ValueError("out must be a contiguous complex128 tensor")
    shape = tuple(field.shape)
    n_cfg, nt, lz, ly, lx = shape[:5]
    dtype = C128 if field.dtype == torch.complex128 else C64
    moms = np.ascontiguousarray(np.array(moms, dtype=np.int32).reshape(-1, 3))
    if len(shape) != 7 or shape[-2:] != (12, 12):
        raise ValueError("field shape must be (n_cfg, nt, Lz, Ly, Lx, 12, 12)")
    pr = Props(field.data_ptr(), field.data_ptr(), dtype, MEM_DEVICE, n_cfg, nt, lx, ly, lz, 0, 0, 1)
    op = ContractOpts(FP64, moms.shape[0], moms.ctypes.data, t0, t1, None, SINK_POINT)
    _check(lib.mbc_contract_noalloc(ctypes.byref(pr), term_list.handle, ctypes.byref(op), out.data_ptr(),
                                    _stream_ptr(stream)), "mbc_contract_noalloc")
    return out


def sync_status(stream=None):
    """``mbc_sync_status``: wait for the stream; raises MbcError with
    MBC_ERR_TIMEOUT (5) when a kernel's bounded wait ran out since the last
    report."""
    _check(load().mbc_sync_status(_stream_ptr(stream)), "mbc_sync_status")


def check_wait_timeout(polls: int = 64, stream=None):
    """``mbc_check_wait_timeout``: run a bounded wait that nothing completes
    (the timeout path's test); the next sync_status reports MBC_ERR_TIMEOUT."""
    _check(load().mbc_check_wait_timeout(int(polls), _stream_ptr(stream)), "mbc_check_wait_timeout")


def release_scratch():
    load().mbc_release_scratch()


def timing_enable(on: bool = True):
    """``mbc_timing_enable``: bracket the contraction kernels with CUDA events."""
    load().mbc_timing_enable(1 if on else 0)


def timing_read():
    """``mbc_timing_read``: (summed kernel milliseconds, launches) since the last read."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().mbc_timing_read(ctypes.byref(ms), ctypes.byref(n)), "mbc_timing_read")
    return ms.value, n.value


def kernel_launches() -> int:
    """``mbc_kernel_launches``: cumulative kernel launches of the contraction."""
    return int(load().mbc_kernel_launches())


def fma_probe(precision: int = FP64) -> float:
    """``mbc_fma_probe``: measured FMA throughput (flop/s) of the current device."""
    f = ctypes.c_double()
    _check(load().mbc_fma_probe(precision, ctypes.byref(f)), "mbc_fma_probe")
    return f.value

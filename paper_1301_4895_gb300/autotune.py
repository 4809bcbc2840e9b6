"""Launch-shape autotuner for mbc_contract.

For a set of term lists, a precision and a lattice geometry it times the
candidate launch shapes of the kernels those lists use - sites per CTA of the
FP64 shared-memory kernel, threads per CTA of the mixed one, wave size and
outputs per warp item of the wave kernels - on a bounded sample of the
caller's field (the first time slices of the first configuration), with
CUDA events on the caller's stream, and keeps the fastest. Results are cached
in a JSON file keyed by (lists, precision, geometry, storage type).

The tuner only chooses ``mbc_tune`` fields; every candidate runs the same
kernels on the same data, so all of them produce the same correlators up to
rounding order.
"""
from __future__ import annotations

import itertools
import json
import os
import threading

from . import FP64, contract

_lock = threading.Lock()


def cache_path() -> str:
    p = os.environ.get("MBC_TUNE_CACHE")
    if p:
        return p
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "mbc", "tune.json")


def _key(field, lists, precision) -> str:
    specs = []
    for tl in lists:
        st = tl.stats()
        specs.append([tl.spec["n_p"], tl.spec["n_n"], tl.spec["dirac_dim"], st["n_ops_total"], st["n_comp"]])
    return json.dumps({"lists": specs, "precision": int(precision), "geom": list(field.shape[2:5]),
                       "dtype": str(field.dtype)}, sort_keys=True)


def candidates(lists, precision):
    small = any(tl.spec["dirac_dim"] == 2 for tl in lists)  # nonrelativistic: shared-memory kernels
    large = any(tl.spec["dirac_dim"] == 4 for tl in lists)  # relativistic: wave kernels
    fp64 = precision == FP64
    opt_small = [{"sites_per_cta": s} for s in (2, 4, 8, 12, 16, 20, 24, 32)] if fp64 else \
        [{"threads_per_cta": t} for t in (256, 512, 768, 1024)]
    if not small:
        opt_small = [{}]
    opt_large = [{}]
    if large:
        opt_large = [dict(w, **z, **o) for w, z, o in itertools.product(
            [{}, {"wave_sites": 128}, {"wave_sites": 512}, {"wave_sites": 2048}],
            [{}, {"zchunk": 4}, {"zchunk": 32}], [{}, {"wave_order": 1}] if fp64 else [{}, {"wave_order": 3}])]
    for a, b in itertools.product(opt_small, opt_large):
        yield dict(a, **b)


def _time(field, lists, precision, tune, t1, stream, reps):
    import torch
    s = stream or torch.cuda.current_stream()
    contract(field, lists, precision=precision, t0=0, t1=t1, tune=tune, stream=s)  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        contract(field, lists, precision=precision, t0=0, t1=t1, tune=tune, stream=s)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(field, lists, precision: int = FP64, stream=None, reps: int = 2, sample_slices: int = 1,
             use_cache: bool = True, verbose: bool = False) -> dict:
    """Best ``mbc_tune`` dict for these lists on this field (torch tensor on
    the device). The timing sample is configuration 0, time slices
    [0, sample_slices)."""
    key = _key(field, lists, precision)
    path = cache_path()
    if use_cache:
        with _lock:
            try:
                with open(path) as f:
                    cached = json.load(f)
                if key in cached:
                    return dict(cached[key]["tune"])
            except (OSError, ValueError):
                pass
    sub = field[:1]
    t1 = max(1, min(sample_slices, field.shape[1]))
    best, best_ms = {}, float("inf")
    results = []
    for cand in candidates(lists, precision):
        try:
            ms = _time(sub, lists, precision, cand, t1, stream, reps)
        except Exception as exc:  # a shape the device cannot run (e.g. shared memory)
            results.append((cand, None, str(exc)))
            continue
        results.append((cand, ms, None))
        if ms < best_ms:
            best, best_ms = cand, ms
    if verbose:
        for cand, ms, err in results:
            print(f"  tune {cand}: {'%.3f ms' % ms if ms is not None else err}")
    if use_cache:
        with _lock:
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                try:
                    with open(path) as f:
                        cached = json.load(f)
                except (OSError, ValueError):
                    cached = {}
                cached[key] = {"tune": best, "ms": best_ms}
                tmp = path + f".{os.getpid()}.tmp"
                with open(tmp, "w") as f:
                    json.dump(cached, f, indent=1, sort_keys=True)
                os.replace(tmp, path)
            except OSError:
                pass
    return dict(best)

#!/usr/bin/env python3
"""Benchmark of the recursive multibaryon contraction on GB300.

Default workload: 3He and 4He with nonrelativistic local operators on a
16^3 x 32 lattice of synthetic u = d propagators (complex128, Gaussian
entries times exp(-0.4 t), seed 1). One step = one mbc_contract call over
the whole lattice for both nuclei (blocks, F_- recursion, contraction with L,
zero-momentum site sum). The headline value is FP64; the mixed FP32-product
/ compensated form is reported beside it with its speedup.

Unit: sink-site correlators per second - one unit is the full requested C
tensor of one nucleus at one (configuration, time slice, sink site).

Multi-GPU (torchrun, one rank per GPU): configurations are sharded, rank r
contracts configuration r of the same recipe; no collective touches the data
path (weak scaling). --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (description, nuclei [(n_p, n_n, D, spins)], dims (Lz, Ly, Lx), nt, seed, lam, dtype)
    "nonrel": ("3He + 4He nonrelativistic, 16^3x32, complex128, seed 1, exp(-0.4 t)",
               [(2, 1, 2, None), (2, 2, 2, None)], (16, 16, 16), 32, 1, 0.4, "c128"),
    "deuteron": ("deuteron (pn) nonrelativistic, all 16 components, 4^3x8, complex128, seed 0, exp(-0.5 t)",
                 [(1, 1, 2, None)], (4, 4, 4), 8, 0, 0.5, "c128"),
    "he4rel1": ("4He relativistic, spin component (0,1,0,1), 16^3x32, complex128, seed 2, exp(-0.4 t)",
                [(2, 2, 4, [((0, 1, 0, 1), (0, 1, 0, 1))])], (16, 16, 16), 32, 2, 0.4, "c128"),
    "he4rel": ("4He relativistic, all 1296 spin components, 16^3 x t-subset, complex128, seed 2",
               [(2, 2, 4, None)], (16, 16, 16), 32, 2, 0.4, "c128"),
    "be8": ("8Be relativistic (0,1,2,3,0,1,2,3), 16^3 x t-subset, complex64 storage, seed 4",
            [(4, 4, 4, [((0, 1, 2, 3, 0, 1, 2, 3), (0, 1, 2, 3, 0, 1, 2, 3))])], (16, 16, 16), 32, 4, 0.4, "c64"),
    "batched": ("batched: pn, 3He, 4He nonrel + 4He rel (0,1,0,1), 24^3x48 per configuration, complex64, seed 3",
                [(1, 1, 2, None), (2, 1, 2, None), (2, 2, 2, None), (2, 2, 4, [((0, 1, 0, 1), (0, 1, 0, 1))])],
                (24, 24, 24), 48, 3, 0.4, "c64"),
    "he4two": ("4He nonrelativistic, two quark sources, two sink functions (momenta (0,0,0) and (1,0,0)), "
               "36 sink components x source spins (0,2,0,2), 16^3x32, complex128, seed 5",
               [(2, 2, 2, [(p + q, (0, 2, 0, 2)) for p in ((0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3))
                           for q in ((0, 1), (0, 2), (1, 2), (0, 3), (1, 3), (2, 3))])],
               (16, 16, 16), 32, 5, 0.4, "c128"),
}
# workloads beyond one source and point sinks: quark sources, sink functions,
# sink mode and the number of momenta per (configuration, time slice)
WORKLOAD_OPTS = {"he4two": {"n_src": 2, "n_sinks": 2, "sink": "block", "moms": 2}}
MOMENTA = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nonrel", choices=sorted(WORKLOADS))
    ap.add_argument("--nt", type=int, default=0, help="time slices (0: workload default)")
    ap.add_argument("--cfgs", type=int, default=1, help="configurations per rank")
    ap.add_argument("--precision", default="both", choices=["both", "fp64", "mixed"])
    ap.add_argument("--graph", action="store_true", help="replay each step from a captured CUDA graph")
    ap.add_argument("--sink", default="", choices=["", "point", "block"],
                    help="point sinks (site correlators summed with the phase) or momentum-projected blocks")
    ap.add_argument("--moms", type=int, default=0, help="momenta per (configuration, time slice)")
    ap.add_argument("--list-free", action="store_true",
                    help="term lists without operation arrays (splits regenerated on the GPU)")
    ap.add_argument("--combined", action="store_true",
                    help="contract the workload's nuclei with one list on a shared recursion path (Sec. 7)")
    ap.add_argument("--autotune", action="store_true", help="pick launch shapes with the autotuner first")
    ap.add_argument("--tune", default="", help='fixed launch shape as JSON, e.g. {"wave_sites": 256}')
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-per-config", action="store_true",
                    help="skip the relativistic 4He and 8Be entries reported beside the default line")
    return ap.parse_args()


def shared_path(nuclei):
    """A recursion path on which every nucleus of the workload is the
    nucleus of a prefix: smaller nuclei first, each adding its extra baryons
    in the paper's order (more numerous species first, neutrons on a tie)."""
    path = []
    cp = cn = 0
    for n_p, n_n, _, _ in sorted(nuclei, key=lambda n: n[0] + n[1]):
        dp, dn = n_p - cp, n_n - cn
        if dp < 0 or dn < 0:
            raise SystemExit("the workload's nuclei do not lie on one path")
        first, nf = (0, dp) if dp > dn else (1, dn)
        path += [first] * nf + [1 - first] * (dp + dn - nf)
        cp, cn = n_p, n_n
    return path


def site_flops(st, dirac_dim):
    nxi = 3 * dirac_dim
    n_g2 = 4 if dirac_dim == 4 else 2
    n_blocks = len(set(st["path"]))
    diquark = 3 * nxi * nxi * (2 * n_g2) * 8
    blocks = n_blocks * st["block_size"] * 6 * 8
    recursion = 8 * st["n_ops_total"]
    contraction = 4 * st["n_l_total"]
    return {"recursion": recursion, "blocks": diquark + blocks, "contraction": contraction,
            "total": recursion + diquark + blocks + contraction}


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        import tempfile
        out_dir = os.environ.get("MBC_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"mbc_clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def profiled_traffic(name, sites, sources=("small_kernel.cuh", "device_common.cuh")):
    """DRAM bytes of a kernel from its committed ncu summary (bytes per site
    x sites), or None when the kernel source changed since the counters were
    taken."""
    import hashlib
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    vals = {}
    with open(path) as f:
        for line in f:
            if ":" in line and line.split(":")[0] in ("traffic_bytes_per_site", "kernel_source_sha256_16"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
    h = hashlib.sha256()
    for src in sources:
        with open(os.path.join(ROOT, "paper_1301_4895_gb300", "csrc", src), "rb") as f:
            h.update(f.read())
    if vals.get("kernel_source_sha256_16") != h.hexdigest()[:16] or "traffic_bytes_per_site" not in vals:
        return None
    return float(vals["traffic_bytes_per_site"]) * sites


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def make_field(wl, cfgs, nt, n_src=1):
    import synth
    _, _, dims, _, seed, lam, dt = wl
    return synth.field(seed, max(cfgs) + 1, nt, dims, lam, dtype=np.complex64 if dt == "c64" else np.complex128,
                       cfgs=list(cfgs), n_src=n_src if n_src > 1 else 0)


def cpu_model() -> str:
    """The host CPU as the OS reports it (model name or implementer/part)."""
    try:
        with open("/proc/cpuinfo") as f:
            info = f.read()
    except OSError:
        return "unknown"
    fields = {}
    for line in info.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            fields.setdefault(k.strip(), v.strip())
    if "model name" in fields:
        return fields["model name"]
    # Arm: implementer and part numbers (Neoverse V2 is the Grace core)
    parts = {"0xd4f": "Neoverse V2", "0xd40": "Neoverse V1", "0xd0c": "Neoverse N1", "0xd8e": "Neoverse N3"}
    if "CPU part" in fields:
        part = fields["CPU part"]
        return f"Arm {parts.get(part, 'core')} (implementer {fields.get('CPU implementer', '?')}, part {part})"
    return fields.get("Model", "unknown")


def cpu_baseline(wl, lists_spec, nt_used, budget_s=15.0, max_sites=None):
    """The oracle (O3, plain C with OpenMP) on a bounded sample: whole slabs
    of the same workload until the budget is spent (relativistic or large
    lattices: the first sites of each slab; max_sites caps them)."""
    from oracle import recursion
    _, nuclei, dims, nt, seed, lam, dt = wl
    import synth
    plans = [recursion.Plan(n_p, n_n, D, requests=comps) for (n_p, n_n, D, _), comps in lists_spec]
    v3 = dims[0] * dims[1] * dims[2]
    done = 0
    t_tot = 0.0
    slabs = 0
    for t in range(nt_used):
        slab = synth.slab(seed, 0, t, dims, lam, np.complex64 if dt == "c64" else np.complex128)
        S = slab.reshape(-1, 12, 12).astype(np.complex128)
        n_sites = v3
        if t_tot > 0 and t_tot > budget_s:
            break
        t0 = time.perf_counter()
        for pl in plans:
            if v3 > 4096 or pl.A > 4 or pl.dim == 4:
                n_sites = min(v3, 256 if pl.A <= 4 else 8)
            if max_sites:
                n_sites = min(n_sites, max_sites)
            pl.evaluate(S[:n_sites], batch=16)
            done += n_sites
        t_tot += time.perf_counter() - t0
        slabs += 1
        if t_tot > budget_s:
            break
    cores = os.cpu_count()
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        pass
    omp = os.environ.get("OMP_NUM_THREADS")
    return {"value": done / t_tot, "unit": "sink-site correlators/s", "cores": int(omp) if omp else cores,
            "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{slabs} slab(s) of the workload, {done} site-correlators over all nuclei, O3 plain "
                      f"recursion in C with OpenMP, {t_tot:.1f} s"}


def oracle_plans(lists_spec, n_src):
    """O3 plans of the workload's nuclei; several quark sources take G~ at
    the source and G for the blocks (Sec. 6)."""
    from oracle import gamma, recursion
    plans = []
    for (n_p, n_n, D, _), comps in lists_spec:
        if n_src > 1:
            plans.append(recursion.Plan(n_p, n_n, D, requests=comps, G=gamma.g_tensor_sources(D, n_src),
                                        G_sink=gamma.g_tensor(D)))
        else:
            plans.append(recursion.Plan(n_p, n_n, D, requests=comps))
    return plans


def cpu_baseline_projected(wl, lists_spec, nt_used, moms, n_src, n_sinks, budget_s=15.0):
    """The oracle with momentum-projected blocks (oracle/projection.py) on
    whole slabs of the workload until the budget is spent."""
    from oracle import projection, recursion
    import synth
    _, nuclei, dims, nt, seed, lam, dt = wl
    plans = oracle_plans(lists_spec, n_src)
    done, t_tot, slabs = 0, 0.0, 0
    for t in range(nt_used):
        if n_src > 1:
            S = recursion.source_columns(synth.slab_sources(seed, 0, t, dims, lam, n_src), nuclei[0][2])
        else:
            S = synth.slab(seed, 0, t, dims, lam, np.complex64 if dt == "c64" else np.complex128)
        t0 = time.perf_counter()
        for pl, (nu, _) in zip(plans, lists_spec):
            projection.projected_correlators(pl, S.astype(np.complex128), dims, moms, n_sinks=n_sinks,
                                             dirac_dim=nu[2])
            done += len(moms) // n_sinks
        t_tot += time.perf_counter() - t0
        slabs += 1
        if t_tot > budget_s:
            break
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    omp = os.environ.get("OMP_NUM_THREADS")
    return {"value": done / t_tot, "unit": "momentum-projected correlators/s", "cores": int(omp) if omp else cores,
            "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"{slabs} slab(s) of the workload, {done} correlators over all nuclei, O3 blocks per site, "
                      f"numpy phase sums, O3 recursion on the summed blocks, {t_tot:.1f} s"}


def run_reference(args, wl):
    """--impl reference: the CPU oracle as it stands, on the host's cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import projection, recursion
    import synth
    _, nuclei, dims, nt, seed, lam, dt = wl
    wopt = WORKLOAD_OPTS.get(args.workload, {})
    n_src, n_sinks = wopt.get("n_src", 1), wopt.get("n_sinks", 1)
    block = (args.sink or wopt.get("sink", "point")) == "block"
    moms = tuple(MOMENTA[:args.moms or wopt.get("moms", 1)])
    plans = oracle_plans([(n, n[3]) for n in nuclei], n_src)
    v3 = dims[0] * dims[1] * dims[2]
    if n_src > 1:
        S = recursion.source_columns(synth.slab_sources(seed, 0, 0, dims, lam, n_src), nuclei[0][2]).reshape(-1, 12, 12)
    else:
        slab = synth.slab(seed, 0, 0, dims, lam, np.complex64 if dt == "c64" else np.complex128)
        S = slab.reshape(-1, 12, 12).astype(np.complex128)
    if block:  # one step: every nucleus' projected correlators of one whole slab
        metric = "momentum-projected correlators/s"
        unit_per_step = (len(moms) // n_sinks) * len(plans)
        sample = f"slab t=0 ({v3} sites) per step, momentum-projected blocks, every nucleus of the workload"

        def step():
            for pl, nu in zip(plans, nuclei):
                projection.projected_correlators(pl, S.reshape(dims + (12, 12)), dims, moms, n_sinks=n_sinks,
                                                 dirac_dim=nu[2])
    else:
        metric = "sink-site correlators/s"
        per_step_sites = 1024 if all(p.dim == 2 for p in plans) else 4
        S = S[: min(v3, per_step_sites)]
        unit_per_step = S.shape[0] * len(plans)
        sample = f"{S.shape[0]} sites of slab t=0 per step, every nucleus of the workload"

        def step():
            for pl in plans:
                pl.evaluate(S, batch=16)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt_s = time.perf_counter() - t0
    units = unit_per_step * args.steps
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    val = units / dt_s
    line = {"impl": "reference", "metric": metric, "value": val,
            "unit": metric, "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt_s / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl[0], "units_per_step": int(unit_per_step)},
            "cpu_baseline": {"value": val, "unit": metric, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": val, "unit": metric, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def point_flops_per_site(stats, list_dims):
    """Algorithmic flops per sink site of point-sink lists: recursion (8 per
    operation) and contraction of every list, plus one diquark and one block
    per species and operator type (the blocks of a site do not depend on the
    nucleus, Sec. 2)."""
    fl = [site_flops(st, d) for st, d in zip(stats, list_dims)]
    per_site = sum(f["recursion"] + f["contraction"] for f in fl)
    for d in sorted(set(list_dims)):
        nxi = 3 * d
        species = set()
        bs = 0
        for st, dd in zip(stats, list_dims):
            if dd == d:
                species |= set(st["path"])
                bs = st["block_size"]
        per_site += 3 * nxi * nxi * (2 * (4 if d == 4 else 2)) * 8 + len(species) * bs * 6 * 8
    return per_site


def l1_operand_bound(n_sm, sm_max_mhz):
    """The mixed recursion's operand bound, flop/s: a site-operation (8 flops)
    reads two 8 B FP32 complex operands through the L1 / shared-memory data
    pipe, which delivers one 128 B wavefront per SM clock."""
    return n_sm * 128.0 * sm_max_mhz * 1e6 / 16.0 * 8.0


def roofline_entry(flops_step, steps, kms, ms, launches, peak, probe, kind, kernel, l1_peak=None):
    """ALU roofline of the contraction kernels: algorithmic flops over their
    CUDA-event time (the whole step when no kernel events were recorded).
    l1_peak (mixed precision): the operand bound of l1_operand_bound beside it."""
    t_ms, basis = (kms, "kernel events") if kms > 0 else (ms, "whole step")
    if not (t_ms == t_ms) or t_ms <= 0:
        return None
    ach = flops_step * steps / (t_ms * 1e-3)
    r = {"bound": "alu", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s", "frac": ach / peak,
         "traffic": None, "peak_kind": kind, "measured_fma_peak": probe / 1e12,
         "frac_of_measured_fma": ach / probe, "kernel": kernel, "time_basis": basis,
         "kernel_ms_per_step": t_ms / steps, "launches_timed": launches, "flops_per_step": flops_step}
    if l1_peak:
        r["l1_operand_bound"] = {
            "peak": l1_peak / 1e12, "unit": "TFLOP/s", "frac": ach / l1_peak,
            "kind": "derived: SMs x 128 B/clk (one L1/shared-memory wavefront) x max SM clock / 16 B of FP32 "
                    "complex operands per site-operation x 8 flop; the data pipe, not the FP32 pipe, bounds the "
                    "mixed recursion (ncu: 63 % of a wavefront per SM clock in k_small_ls on the default workload, "
                    "81 % L1/shared throughput in k_large_step_split on 8Be's largest step)"}
    return r


# Configurations of the metric's headline nuclei reported beside the default
# line: (workload, what the entry covers, oracle sample sites, profile of the
# dominant kernels' DRAM traffic per site: FP64, mixed).
PER_CONFIG = {
    "he4rel_all_components": (
        "he4rel", "4He relativistic, all 1296 spin components (Table 1: 531,321,120 operations per site), "
        "one 16^3 slab (t = 0) of the 16^3x32 lattice, complex128, seed 2", 8,
        ("k_large_step_fp64_he4rel_all_16x16x16x1.md", "k_large_step_split_mixed_he4rel_all_16x16x16x1.md")),
    "be8": (
        "be8", "8Be relativistic (0,1,2,3,0,1,2,3) (Tables 1, 5: 448,496,928 operations per site), one 16^3 slab "
        "(configuration 0, t = 0) of the 16^3x32 x 12 lattice, complex64 storage, seed 4", 8,
        ("k_large_step_fp64_be8_16x16x16x1.md", "k_large_step_split_mixed_be8_16x16x16x1.md")),
}


def per_config_entry(mbc, torch, dev, name, peaks, n_sm, probes, warmup=3, steps64=1, steps_mx=3):
    """FP64 and mixed throughput of one headline configuration on one slab
    (the full lattices scale linearly in slabs: no work is shared between
    slabs), with its roofline, clocks, host-buffer e2e (mixed) and the oracle
    on a bounded sample of the same slab."""
    key, what, cpu_sites, prof = PER_CONFIG[name]
    wl = WORKLOADS[key]
    _, nuclei, dims, _, _, _, _ = wl
    nt = 1
    lists = [mbc.build_term_list(n_p, n_n, D, spins=spins) for (n_p, n_n, D, spins) in nuclei]
    stats = [tl.stats() for tl in lists]
    field_np = make_field(wl, [0], nt)
    field = torch.from_numpy(field_np).to(dev)
    stream = torch.cuda.Stream(dev)
    v3 = dims[0] * dims[1] * dims[2]
    units = v3 * nt * len(nuclei)
    flops_step = point_flops_per_site(stats, [n[2] for n in nuclei]) * v3 * nt
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak = {0: n_sm * 2 * 2 * sm_max * 1e6, 1: n_sm * 128 * 2 * sm_max * 1e6}
    kinds = {0: f"FP64 vector, derived: {n_sm} SMs x 2 DFMA/clk x max SM clock",
             1: f"FP32 vector, derived: {n_sm} SMs x 128 FFMA/clk x max SM clock"}
    kernels = {0: "k_large_step<FP64>", 1: "k_large_step_split"}
    # the launch shape changes the step kernels' traffic: the launch code is hashed too
    src = ("large_kernel.cuh", "mixed_common.cuh", "device_common.cuh", "contract.cu")
    entry = {"workload": what, "units_per_step": units, "sites_per_step": v3 * nt, "n_ops": [st["n_ops_total"] for st in stats],
             "unit": "sink-site correlators/s", "warmup": warmup, "steps": {"fp64": steps64, "mixed": steps_mx}}
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        for prec, steps in ((0, steps64), (1, steps_mx)):
            for _ in range(warmup):
                mbc.contract(field, lists, precision=prec, stream=stream)
            torch.cuda.synchronize(dev)
            mbc.timing_enable(True)
            mbc.timing_read()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                mbc.contract(field, lists, precision=prec, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            kms, launches = mbc.timing_read()
            mbc.timing_enable(False)
            roof = roofline_entry(flops_step, steps, kms, ms, launches, peak[prec], probes[prec], kinds[prec],
                                  kernels[prec], l1_operand_bound(n_sm, sm_max) if prec == 1 else None)
            if roof is not None:
                roof["traffic"] = profiled_traffic(prof[prec], v3 * nt, src)
                roof["traffic_note"] = ("DRAM bytes of the step kernel per step (all its launches), from the "
                                        "committed ncu summary scaled by sites; null if the kernel changed since")
            entry["fp64" if prec == 0 else "mixed"] = {"value": units * steps / (ms * 1e-3), "ms_per_step": ms / steps,
                                                       "roofline": roof}
    entry["clocks"] = clk.summary()
    entry["mixed"]["speedup_vs_fp64"] = entry["mixed"]["value"] / entry["fp64"]["value"]
    # end to end through the public API with host buffers (pinned), mixed
    pinned = torch.empty(field_np.shape, dtype=field.dtype, pin_memory=True)
    pinned.copy_(torch.from_numpy(field_np))
    host = pinned.numpy()
    mbc.contract(host, lists, precision=1)
    t0 = time.perf_counter()
    res = mbc.contract(host, lists, precision=1)
    _ = complex(res.reshape(-1)[0])
    dt_s = time.perf_counter() - t0
    entry["e2e"] = {"value": units / dt_s, "unit": "sink-site correlators/s", "precision": "mixed", "steps": 1,
                    "h2d_bytes_per_step": int(field_np.nbytes), "d2h_bytes_per_step": int(res.nbytes)}
    entry["cpu_baseline"] = cpu_baseline(wl, [(n, tl.components()) for n, tl in zip(nuclei, lists)], nt,
                                         budget_s=8.0, max_sites=cpu_sites)
    for tl in lists:
        tl.free()
    del field
    torch.cuda.empty_cache()
    return entry


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)
    import torch
    import paper_1301_4895_gb300 as mbc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    desc, nuclei, dims, nt_full, seed, lam, dt = wl
    nt = args.nt or nt_full
    if args.workload in ("he4rel", "be8") and not args.nt:
        nt = 1  # one time slice: 4096 sinks
    wopt = WORKLOAD_OPTS.get(args.workload, {})
    n_src, n_sinks = wopt.get("n_src", 1), wopt.get("n_sinks", 1)
    sink = args.sink or wopt.get("sink", "point")
    n_mom = args.moms or wopt.get("moms", 1)
    if n_mom % n_sinks or n_mom > len(MOMENTA):
        raise SystemExit("momenta must fill whole groups of sink functions")
    moms = tuple(MOMENTA[:n_mom])
    sink_mode = mbc.SINK_BLOCK_MOMENTUM if sink == "block" else mbc.SINK_POINT
    if args.combined:
        if len({n[2] for n in nuclei}) != 1:
            raise SystemExit("--combined needs one operator type")
        lists = [mbc.build_combined([dict(n_p=a, n_n=b, spins=sp) for a, b, _, sp in nuclei], nuclei[0][2],
                                    path=shared_path(nuclei))]
        list_dims = [nuclei[0][2]]
    else:
        lists = [mbc.build_term_list(n_p, n_n, D, spins=spins, list_free=args.list_free, n_sources=n_src,
                                     n_sinks=n_sinks) for (n_p, n_n, D, spins) in nuclei]
        list_dims = [n[2] for n in nuclei]
    stats = [tl.stats() for tl in lists]
    field_np = make_field(wl, range(rank * args.cfgs, (rank + 1) * args.cfgs), nt, n_src)
    v3 = dims[0] * dims[1] * dims[2]
    field = torch.from_numpy(field_np).to(dev)
    stream = torch.cuda.Stream(dev)
    if sink == "block":  # one unit: a nucleus' correlator tensor at one (cfg, t, momentum group)
        units_per_step = nt * (n_mom // n_sinks) * len(nuclei) * args.cfgs
        metric = "momentum-projected correlators/s"
    else:  # one unit: a nucleus' correlator tensor at one (cfg, t, sink site)
        units_per_step = v3 * nt * len(nuclei) * args.cfgs
        metric = "sink-site correlators/s"
    tunes = {0: None, 1: None}
    if args.tune:
        tunes = {0: json.loads(args.tune), 1: json.loads(args.tune)}
    if args.autotune:
        from paper_1301_4895_gb300.autotune import autotune
        for p in (0, 1):
            tunes[p] = autotune(field, lists, precision=p, stream=stream)
    graphs = {}

    def step(precision):
        if not args.graph:
            return mbc.contract(field, lists, precision=precision, stream=stream, tune=tunes[precision], moms=moms,
                                sink=sink_mode)
        if precision not in graphs:
            with torch.cuda.stream(stream):
                out = mbc.contract(field, lists, precision=precision, stream=stream, tune=tunes[precision], moms=moms,
                                   sink=sink_mode)
            stream.synchronize()
            g = torch.cuda.CUDAGraph()
            n0 = mbc.kernel_launches()
            with torch.cuda.graph(g, stream=stream):
                mbc.contract(field, lists, precision=precision, stream=stream, tune=tunes[precision], out=out,
                             moms=moms, sink=sink_mode)
            graphs[precision] = (g, out, mbc.kernel_launches() - n0)
        g, out, _ = graphs[precision]
        with torch.cuda.stream(stream):
            g.replay()
        return out

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(precision, steps, warmup):
        for _ in range(warmup):
            step(precision)
        torch.cuda.synchronize(dev)
        mbc.timing_enable(True)
        mbc.timing_read()
        barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        n0 = mbc.kernel_launches()
        e0.record(stream)
        for _ in range(steps):
            out = step(precision)
        e1.record(stream)
        launch_count[precision] = mbc.kernel_launches() - n0
        if args.graph:  # each replay runs the kernels captured from one call
            launch_count[precision] = graphs[precision][2] * steps
        torch.cuda.synchronize(dev)
        barrier()
        ms = e0.elapsed_time(e1)
        kms, launches = mbc.timing_read()
        mbc.timing_enable(False)
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        if world > 1:
            import torch.distributed as dist
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item()), kms, launches, out

    nan = float("nan")
    launch_count = {0: 0, 1: 0}
    outs = {}
    with ClockSampler(local) as clk:
        if args.precision in ("both", "fp64"):
            ms64, k64, n64, outs[0] = timed(0, args.steps, args.warmup)
        else:
            ms64, k64, n64 = nan, 0.0, 0
        if args.precision in ("both", "mixed"):
            msmx, kmx, nmx, outs[1] = timed(1, args.steps, args.warmup)
        else:
            msmx, kmx, nmx = nan, 0.0, 0
    clocks = clk.summary()
    primary = 0 if args.precision in ("both", "fp64") else 1
    # the one exchange of the sharded path, after the timed region: every
    # rank's per-slab correlators gathered in slab order (shard.gather_slabs)
    exchange = None
    if world > 1:
        from paper_1301_4895_gb300.shard import gather_slabs
        res_local = outs[primary].cpu().numpy()  # (cfgs, n_lists, nt, n_mom', n_comp)
        part = {(rank * args.cfgs + c, t): res_local[c, :, t] for c in range(args.cfgs) for t in range(nt)}
        full = gather_slabs(part, world * args.cfgs, nt, res_local.shape[1:2] + res_local.shape[3:])
        exchange = {"kind": "gather of per-slab correlators after the timed region", "bytes": int(full.nbytes)}

    # end to end through the public API with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        pinned = torch.empty(field_np.shape, dtype=field.dtype, pin_memory=True)
        pinned.copy_(torch.from_numpy(field_np))
        host = pinned.numpy()
        for _ in range(max(1, args.warmup)):
            mbc.contract(host, lists, precision=primary, moms=moms, sink=sink_mode)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            res = mbc.contract(host, lists, precision=primary, moms=moms, sink=sink_mode)
            _ = complex(res.reshape(-1)[0])  # the step's result read on the host
        dt_s = time.perf_counter() - t0
        tt = torch.tensor([dt_s], dtype=torch.float64, device=dev)
        if world > 1:
            import torch.distributed as dist
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        dt_s = float(tt.item())
        e2e = {"value": units_per_step * world * args.steps / dt_s, "unit": metric,
               "h2d_bytes_per_step": int(field_np.nbytes), "d2h_bytes_per_step": int(res.nbytes)}

    if rank != 0:
        return 0

    value64 = units_per_step * world * args.steps / (ms64 * 1e-3)
    value_mx = units_per_step * world * args.steps / (msmx * 1e-3)
    value = value64 if primary == 0 else value_mx
    # roofline of the dominant kernel (the contraction kernel; FP64 pipe)
    if sink == "block":
        # per site: blocks of one sink function and their phase-weighted sums
        # over the momenta; per (cfg, t, group): recursion and contraction
        per_site = per_item = 0
        for st, d in zip(stats, list_dims):
            bs_site = st["block_size"] // n_sinks
            nxi = 3 * d * n_src
            n_blocks = len(set(st["path"]))
            per_site += 3 * nxi * nxi * (2 * (4 if d == 4 else 2)) * 8 + n_blocks * bs_site * (6 * 8 + n_mom * 8)
            per_item += 8 * st["n_ops_total"] + 4 * st["n_l_total"]
        flops_step = (per_site * v3 + per_item * (n_mom // n_sinks)) * nt * args.cfgs
    else:
        flops_step = point_flops_per_site(stats, list_dims) * v3 * nt * args.cfgs
    peaks = measured_peaks()
    probe64 = mbc.fma_probe(0)
    probe32 = mbc.fma_probe(1)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    nominal64 = n_sm * 2 * 2 * sm_max * 1e6  # 2 DFMA / clk / SM (1.25 TFLOP/s class), 2 flop each
    nominal32 = n_sm * 128 * 2 * sm_max * 1e6
    has_small = any(n[2] == 2 for n in nuclei)
    has_large = any(n[2] == 4 for n in nuclei)
    kname = {0: " + ".join(k for k, on in (("k_small<FP64>", has_small), ("k_large_step<FP64>", has_large)) if on),
             1: " + ".join(k for k, on in (("k_small_ls<Mixed>", has_small),
                                            ("k_large_step_gen" if args.list_free else "k_large_step_split", has_large))
                           if on)}
    if sink == "block" or n_src > 1 or args.list_free:  # wave kernels only
        kname = {0: "k_large_step<FP64>", 1: "k_large_step_gen" if args.list_free else "k_large_step_split"}
        if sink == "block":
            kname = {p: "k_project_blocks + " + k for p, k in kname.items()}

    def roofline(kms, ms, launches, peak, probe, kind, prec):
        return roofline_entry(flops_step, args.steps, kms, ms, launches, peak, probe, kind, kname[prec],
                              l1_operand_bound(n_sm, sm_max) if prec == 1 else None)

    roof64 = roofline(k64, ms64, n64, nominal64, probe64,
                      f"FP64 vector, derived: {n_sm} SMs x 2 DFMA/clk x max SM clock", 0)
    roof_mx = roofline(kmx, msmx, nmx, nominal32, probe32,
                       f"FP32 vector, derived: {n_sm} SMs x 128 FFMA/clk x max SM clock", 1)
    roof = roof64 if primary == 0 else roof_mx
    if args.workload == "nonrel" and not has_large and not args.combined and not args.graph:
        note = ("DRAM bytes per launch (one launch per step) from the committed ncu summary, "
                "scaled from 65,536 to the step's sites")
        for r, name, srcs in ((roof64, "k_small_fp64_he3_he4_16x16x16x16.md", ("small_kernel.cuh", "device_common.cuh")),
                              (roof_mx, "k_small_ls_mixed_he3_he4_16x16x16x16.md",
                               ("small_ls_kernel.cuh", "mixed_common.cuh", "device_common.cuh"))):
            if r is not None:
                r["traffic"] = profiled_traffic(name, v3 * nt * args.cfgs, srcs)
                r["traffic_note"] = note
    line = {
        "metric": metric, "value": value, "unit": metric, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": (ms64 if primary == 0 else msmx) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if primary == 0 else "f32+f64", "data": "synthetic",
        "config": {"workload": desc, "nuclei": [f"({n[0]},{n[1]}) D={n[2]}" for n in nuclei],
                   "sites_per_step": v3 * nt * args.cfgs, "units_per_step": units_per_step,
                   "configurations_per_rank": args.cfgs, "graph": bool(args.graph),
                   "combined_path": stats[0]["path"] if args.combined else None,
                   "list_free": bool(args.list_free), "list_bytes": [st["op_bytes"] for st in stats],
                   "tune": {"fp64": tunes[0], "mixed": tunes[1]},
                   "l2": "inputs larger than L2 (field %.0f MB)" % (field_np.nbytes / 2 ** 20),
                   "parallelism": f"configurations sharded over {world} GPU(s)", "exchange": exchange},
        "roofline": roof,
        "fp64": {"value": value64, "ms_per_step": ms64 / args.steps, "roofline": roof64},
        "mixed": {"value": value_mx, "ms_per_step": msmx / args.steps, "speedup_vs_fp64": value_mx / value64,
                  "dtype": "f32 products, Kahan-compensated f32 accumulation, f64 contraction and site sums", "roofline": roof_mx},
        "clocks": clocks,
        "e2e": e2e,
        # kernels the library launched in the timed region(s) (graph replays
        # launch the captured kernels without passing through the library)
        "gpu_launches": int(launch_count[0] + launch_count[1]),
        "gpu_launches_per_step": {"fp64": launch_count[0] / args.steps, "mixed": launch_count[1] / args.steps},
        "n_ops": [st["n_ops_total"] for st in stats],
    }
    if not args.no_per_config and world == 1 and args.workload == "nonrel" and not (args.combined or args.graph):
        line["per_config"] = {name: per_config_entry(mbc, torch, dev, name, peaks, n_sm, {0: probe64, 1: probe32})
                              for name in PER_CONFIG}
    if not args.no_cpu_baseline and world == 1:  # the oracle baseline is a single-GPU figure
        if sink == "block":
            line["cpu_baseline"] = cpu_baseline_projected(wl, [(n, tl.components()) for n, tl in zip(nuclei, lists)],
                                                          nt, moms, n_src, n_sinks)
        else:
            if args.combined:  # one list, one part per nucleus: each nucleus' own components
                comps = lists[0].components()
                spec = []
                for part in lists[0].parts():
                    a_ = part["n_p"] + part["n_n"]
                    nu = next(n for n in nuclei if n[0] == part["n_p"] and n[1] == part["n_n"])
                    spec.append((nu, [(snk[:a_], src[:a_]) for snk, src in comps[part["c0"]:part["c1"]]]))
            else:
                spec = [(n, tl.components()) for n, tl in zip(nuclei, lists)]
            line["cpu_baseline"] = cpu_baseline(wl, spec, nt)
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

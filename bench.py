"""Benchmark: aggregate risk analysis on one GB300 (or N independent ranks).

One step = one pass of the hot path over the workload: the YLT forward
(lookup, financial terms, ELT sum, occurrence terms, FP64 aggregate and
aggregate terms for every layer and trial) and the metrics (mean, PML and
TVaR per layer). Default workload: 1,000,000 trials x 1,000 events over a
2,000,000-event catalogue, one layer of 16 ELTs with 20,000 non-zero
lognormal(12, 2) losses each (synthetic, seeded).

Metric: trial-events x ELTs per second (sum_t K_t * sum_j |E_j| per step /
step time), plus ms per 1M-trial YLT and the roofline fraction of the
forward kernel. After the headline line's timed region, the batching (c2),
differentiation (c3) and precision (c4) workloads are timed too and reported
in its `workloads` record (--workloads none skips them); they are
single-GPU figures, timed at N = 1 only.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config c1]
                  [--variant auto|plain|batched|fp64|skip|sparse]
                  [--impl ours|reference] [--workloads c2,c3,c4|none]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
CONFIG_TEXT = {
    "c1": "1,000,000 trials x 1,000 events, catalogue 2,000,000, 1 layer x 16 ELTs (20,000 non-zero lognormal(12,2) "
          "losses each), occR 1e5 occL 5e6 aggR 1e6 aggL 2e7, PML/TVaR at 0.99",
    "c1u": "config c1 with aggR 9e7 aggL 5e7 (aggregate terms straddle the median aggregate)",
    "c0": "10,000 trials x 1,000 events, catalogue 100,000, 1 layer x 3 ELTs",
    "c2": "1,000,000 trials of clamp(Poisson(1000),200,2000) events (CSR), 64 layers x U{1..32} ELTs from a pool of 256",
    "c4": "1,000,000 trials x 1,000 events, 128 layers x U{4..32} ELTs from a pool of 512, lognormal(13,2.5)",
    "c3": "c1's YET and 16 ELTs, 8 layers of 8 ELTs; step = forward + EL/TVaR_0.99 + their gradients w.r.t. "
          "OccR, OccL, AggR, AggL and the 16 ELT multipliers (adjoint)",
}
VARIANT_KERNEL = {"plain": "ylt_plain", "batched": "ylt_batched", "fp64": "ylt_skip64", "skip": "ylt_skip",
                  "sparse": "ylt_sparse"}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def rank_max(value: float, dist, device=None) -> float:
    """Max of a per-rank scalar over all ranks (the step time that counts is
    the slowest rank's); identity without a process group."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, n_ranks: int, seconds: float) -> float:
    """Units all ranks processed over the slowest rank's time (weak scaling:
    every rank runs the same workload on its own GPU)."""
    return n_ranks * units_per_rank / seconds


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    try:
        with open(PEAKS_FILE) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


KERNEL_SOURCES = {"ylt_plain": "ylt_plain.cu", "ylt_skip": "ylt_skip.cu", "ylt_batched": "ylt_batched.cu",
                  "ylt_skip64": "ylt_skip64.cu", "ylt_sparse": "ylt_sparse.cu", "metrics": "metrics.cu",
                  "adjoint_group": "adjoint_group.cu"}


def kernel_source_hash(kernel: str) -> str:
    """Hash of the kernel's own source file and the shared device header."""
    h = hashlib.sha256()
    for f in (KERNEL_SOURCES[kernel], "art_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1308_2572_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str, profiles_dir: str = None):
    """DRAM bytes per launch from the committed ncu record
    profiles/<kernel>_<workload>.json ({"source_hash", "dram_bytes_per_launch",
    ...}), if it was taken on the current kernel sources; else None."""
    path = os.path.join(profiles_dir or os.path.join(ROOT, "profiles"), f"{kernel}_{workload}.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("source_hash") != kernel_source_hash(kernel):
        return None
    v = rec.get("dram_bytes_per_launch")
    return float(v) if v is not None else None


def layer_groups(port, with_layers: bool = False):
    """The library's layer groups (consecutive layers while a group has at
    most 8 layers and at most 32 distinct ELTs), as ELT-id lists (with
    with_layers, as (ELT ids, layer ids) pairs)."""
    groups, uni, lay = [], [], []
    for j in range(port.n_layers):
        elts = [int(e) for e in port.layer_elt_ids[port.layer_elt_off[j]:port.layer_elt_off[j + 1]]]
        merged = uni + [e for e in elts if e not in uni]
        if lay and (len(lay) >= 8 or len(merged) > 32):
            groups.append((uni, lay))
            uni, lay, merged = [], [], list(elts)
        uni, lay = merged, lay + [j]
    if lay:
        groups.append((uni, lay))
    return groups if with_layers else [g for g, _ in groups]


def occurrence_groups(port, per: int = 8):
    """The skip variant's occurrence groups: runs of up to 8 (the all-FP64
    variant's: 4) consecutive layers, as lists of layer ids."""
    return [list(range(j, min(j + per, port.n_layers))) for j in range(0, port.n_layers, per)]


def occurrence_density(port, layers) -> float:
    """Fraction of catalogue events with a positive occurrence loss in any of
    the given layers (the density of the skip variant's per-call bitmap).
    Accounting only: FP64 on the host."""
    rows = None
    for j in layers:
        e = port.layer_elt_ids[port.layer_elt_off[j]:port.layer_elt_off[j + 1]]
        nz = np.any(port.elt_losses[e] != 0, axis=0)
        rows = nz if rows is None else (rows | nz)
    idx = np.nonzero(rows)[0]
    hit = np.zeros(idx.size, dtype=bool)
    for j in layers:
        if not port.occ_lim[j] > 0:
            continue
        e = port.layer_elt_ids[port.layer_elt_off[j]:port.layer_elt_off[j + 1]]
        x = np.zeros(idx.size)
        for k in e:
            l = port.elt_losses[k, idx].astype(np.float64)
            x += np.clip(float(port.elt_mult[k]) * l - float(port.elt_ded[k]), 0.0, float(port.elt_lim[k]))
        hit |= x > float(port.occ_ret[j])
    return float(hit.sum()) / port.catalogue_size


def _pad(n: int) -> int:
    return 4 if n <= 4 else (8 if n <= 8 else (16 if n <= 16 else (24 if n <= 24 else 32)))


def _sec(nbytes) -> int:
    return 32 * -(-int(nbytes) // 32)


def csr_build_used(port, layouts: int) -> bool:
    """Whether the library builds the skip variant's occurrence tables from
    the CSR of the non-zero losses: whenever the portfolio holds it
    (ART_LAYOUT_SPARSE). A layer listed out of ascending ELT order has the
    events with three or more of its entries re-summed from its per-layer
    row; the accounting leaves those rare rows out."""
    from paper_1308_2572_gb300 import art
    return bool(layouts & art.ART_LAYOUT_SPARSE)


def builds_from_csr(port, layouts: int, variant: str) -> bool:
    """Whether this variant's occurrence tables come from the CSR (the skip
    and all-FP64 builds, whenever the portfolio holds it)."""
    return variant in ("skip", "fp64") and csr_build_used(port, layouts)


def algorithmic_bytes(w, variant: str, l2_bytes: float = 126e6, csr_build: bool = False):
    """What one forward launch set moves and reads, for the roofline.

    s8d: the per-unit figure -- 4 B per event id (plus 8 B per CSR offset)
      and the 32-byte sectors every table read touches (32 * ceil(row / 32)
      per row read; 32 B of offsets plus 8 B per entry for the CSR), plus the
      YLT written; for the skip and all-FP64 variants, the rows read are
      those of the per-call occurrence-loss tables X, plus their build pass
      (per-layer tables read once, X and the bitmaps written).
    compulsory: the least DRAM traffic of the pass -- ids, offsets and YLT
      once, plus every distinct table row a pass can touch read once (for the
      skip and all-FP64 variants: the build pass; X is then gathered from L2).
    l2: the L2 sector traffic -- the id stream, the sectors the table reads
      touch and the build pass.
    table_bytes: the largest table the per-event reads gather from (X for the
      skip and all-FP64 variants: (C + 1) rows of LP entries); l2_resident
      says whether it fits the L2 (l2_bytes), in which case its gathers are
      L2 traffic, not DRAM traffic.
    lookups_performed: table entries the kernels read per launch set (the
      skip and all-FP64 variants: one per (catalogue event, layer ELT) in the
      build plus one X row per gathered event; the others: per occurrence).
    csr_build: the skip and all-FP64 builds read the CSR of the non-zero
      losses (per group: the C + 1 offsets and every 8-byte entry) instead of
      the per-layer tables; the lookups of the build are then its entries.
    """
    port, yet = w.portfolio, w.yet
    n_events = yet.n_events
    ids = 4 * n_events + (8 * (yet.n_trials + 1) if yet.trial_off is not None else 0)
    ylt = 8 * yet.n_trials * port.n_layers
    C = port.catalogue_size
    touched_frac = 1.0 - np.exp(-n_events / C)
    elts_total = float(port.elts_per_layer().sum())
    if variant in ("skip", "fp64"):
        # one streamed pass over the per-layer tables writes each occurrence
        # group's table X [C + 1][LP] and its bitmap, then per group and
        # event an id and, where X is non-zero, one sector of X (the all-FP64
        # variant: 8-byte entries of X in groups of 4 layers)
        L = port.n_layers
        per = 4 if variant == "fp64" else 8
        lp = 1 if L <= 1 else (2 if L <= 2 else (4 if (L <= 4 or per == 4) else 8))
        xb = 8 if variant == "fp64" else 4
        groups = occurrence_groups(port, per)
        dens = [occurrence_density(port, lays) for lays in groups]
        gathered = sum(n_events * d for d in dens)
        reads = sum(n_events * d * _sec(xb * lp) for d in dens)
        nnz = float((port.elt_losses != 0).sum())
        if csr_build:
            build = len(groups) * (4.0 * (C + 1) + 8.0 * nnz + (C + 1) * xb * lp + C / 8)
            build_lookups = len(groups) * nnz
        else:
            build = float(sum(4 * _pad(int(n)) for n in port.elts_per_layer())) * C + len(groups) * (
                (C + 1) * xb * lp + C / 8)
            build_lookups = C * elts_total
        n_groups = len(groups)
        table = float((C + 1) * xb * lp)
        # FP64 operations of the all-FP64 variant: its CSR build costs an FMA
        # per non-zero loss and an add per (loss, layer holding it); the trial
        # pass adds the FP64 occurrence losses as integers (no FP64 operation)
        flops = 2.0 * nnz + nnz * elts_total / port.n_elt
        out = {"s8d": n_groups * ids + ylt + build + reads, "compulsory": n_groups * ids + ylt + build,
               "l2": n_groups * ids + build + reads, "table_bytes": table, "l2_resident": table <= l2_bytes,
               "lookups_performed": build_lookups + gathered}
        if variant == "fp64":
            out["fp64_flops"] = flops
        return out
    if variant == "sparse":
        nnz = float((port.elt_losses != 0).sum())
        nnz_per_event = nnz / C
        csr = 4 * (C + 1) + 8 * nnz
        reads = n_events * (32 + 8 * nnz_per_event)
        return {"s8d": ids + ylt + reads, "compulsory": ids + ylt + csr * touched_frac, "l2": ids + reads,
                "table_bytes": csr, "l2_resident": csr <= l2_bytes, "lookups_performed": n_events * nnz_per_event}
    if variant == "plain":
        rows = [4 * _pad(int(n)) for n in port.elts_per_layer()]
        reads = float(sum(_sec(r) for r in rows)) * n_events
        table = float(sum(rows)) * C
        n_launch = port.n_layers
        looked = n_events * elts_total
        biggest = float(max(rows)) * C
    else:
        epl = 1
        while 32 * epl < port.n_elt:
            epl *= 2
        rowb = 32 * epl * (8 if variant == "fp64" else 4)
        reads = float(_sec(rowb)) * n_events
        table = biggest = float(rowb) * C
        n_launch = 1
        looked = n_events * 32.0 * epl
    return {"s8d": n_launch * ids + ylt + reads, "compulsory": n_launch * ids + ylt + table * touched_frac,
            "l2": n_launch * ids + reads, "table_bytes": biggest, "l2_resident": biggest <= l2_bytes,
            "lookups_performed": looked}


def roofline(ab: dict, secs: float, hbm_gbs: float, l2_gbs=None, fp64_gflops=None) -> dict:
    """The bound a forward launch set runs against, from its accounting (see
    algorithmic_bytes) and its measured time.

    A gathered table that fits L2 (the skip and all-FP64 variants'
    occurrence tables): t* = max(compulsory DRAM bytes / HBM peak, L2 sector
    bytes / probed L2 gather rate); a table larger than L2: every sector read
    counts as DRAM traffic, t* = per-unit bytes / HBM peak. Where the launch
    set does FP64 arithmetic (the all-FP64 variant's build) and the probed
    FP64 add rate is given, its FP64 operations / that rate is a third term.
    The largest term names the bound ("hbm", "l2" or "alu") and gives
    achieved and peak, so frac = achieved / peak = t* / t. Without the L2
    probe the L2 term is left out. Beside the bound the line keeps the HBM
    fraction by the compulsory DRAM bytes alone.
    """
    gb = lambda b: b / secs / 1e9
    out = {"hbm_frac_by_dram_bytes": gb(ab["compulsory"]) / hbm_gbs,
           "algorithmic_bytes_per_launch": ab["s8d"], "compulsory_bytes_per_launch": ab["compulsory"],
           "l2_sector_bytes_per_launch": ab["l2"], "l2_sector_gbs": gb(ab["l2"]),
           "gathered_table_bytes": ab["table_bytes"], "gathered_table_fits_l2": bool(ab["l2_resident"])}
    terms = {}
    if ab["l2_resident"]:
        terms["hbm"] = (ab["compulsory"] / (hbm_gbs * 1e9),
                        dict(achieved=gb(ab["compulsory"]), peak=hbm_gbs, unit="GB/s",
                             peak_source="hbm_gbs (copy bandwidth)"))
        if l2_gbs:
            terms["l2"] = (ab["l2"] / (l2_gbs * 1e9),
                           dict(achieved=gb(ab["l2"]), peak=l2_gbs, unit="GB/s",
                                peak_source="probed random 32-byte L2 gather rate (art_probe)"))
    else:
        terms["hbm"] = (ab["s8d"] / (hbm_gbs * 1e9),
                        dict(achieved=gb(ab["s8d"]), peak=hbm_gbs, unit="GB/s", peak_source="hbm_gbs (copy bandwidth)"))
    if ab.get("fp64_flops") and fp64_gflops:
        out["fp64_flops_per_launch"] = ab["fp64_flops"]
        terms["alu"] = (ab["fp64_flops"] / (fp64_gflops * 1e9),
                        dict(achieved=ab["fp64_flops"] / secs / 1e9, peak=fp64_gflops, unit="GFLOP/s",
                             peak_source="probed FP64 add rate (art_probe)"))
    bound = max(terms, key=lambda k: terms[k][0])
    out["t_star_ms"] = terms[bound][0] * 1e3
    out.update(bound=bound, **terms[bound][1])
    out["frac"] = out["achieved"] / out["peak"]
    return out


def first_layers(w, n: int):
    """The workload with only its first n layers (smaller profiling cases of
    the multi-layer kernels: the same occurrence-group shapes, fewer groups)."""
    import dataclasses
    port = w.portfolio
    n = min(n, port.n_layers)
    off = port.layer_elt_off[:n + 1].copy()
    sub = dataclasses.replace(port, layer_elt_off=off, layer_elt_ids=port.layer_elt_ids[:off[-1]].copy(),
                              occ_ret=port.occ_ret[:n].copy(), occ_lim=port.occ_lim[:n].copy(),
                              agg_ret=port.agg_ret[:n].copy(), agg_lim=port.agg_lim[:n].copy())
    return dataclasses.replace(w, portfolio=sub)


def synthetic_ylt(torch, L: int, T: int, dev, seed: int = 1308):
    """A seeded YLT [L][T] shaped like the pool workloads' (lognormal
    aggregate losses, a quarter of the trials without loss, a layer-dependent
    share of 0-30% of the trials at the layer's aggregate cap), for timing
    the metrics kernels alone."""
    g = torch.Generator(device=dev).manual_seed(seed)
    y = torch.empty((L, T), dtype=torch.float64, device=dev)
    y.log_normal_(16.0, 1.5, generator=g)
    share = torch.linspace(0.0, 0.3, L, dtype=torch.float64, device=dev)
    head = torch.sort(y[:, :min(T, 50000)], dim=1).values
    idx = ((1.0 - share) * (head.shape[1] - 1)).long()
    cap = head[torch.arange(L, device=dev), idx]
    torch.minimum(y, cap[:, None], out=y)
    y[:, ::4] = 0.0
    return y


def run_metrics_only(args):
    """art_metrics alone on a synthetic YLT of --layers x --trials (default
    128 x 1,000,000) at --probs: ms per call, and GB/s per full read."""
    import torch
    from paper_1308_2572_gb300 import art
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    L, T = args.layers or 128, args.trials or 1_000_000
    probs = [float(x) for x in args.probs.split(",")]
    y = synthetic_ylt(torch, L, T, dev)
    n_p = len(probs)
    mean = torch.empty(L, dtype=torch.float64, device=dev)
    pml = torch.empty((L, n_p), dtype=torch.float64, device=dev)
    tvar = torch.empty((L, n_p), dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        art.art_metrics(y, T, L, probs, mean, pml, tvar)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        art.art_metrics(y, T, L, probs, mean, pml, tvar)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"metrics_only": True, "layers": L, "trials": T, "probs": probs, "ms_per_call": ms,
                      "ylt_gbs_per_full_read": L * T * 8 / (ms * 1e-3) / 1e9}), flush=True)
    return 0


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on the host cores, on a
    bounded sample of the workload per step."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1308_2572_gb300 import workloads
    sample_trials = args.ref_trials
    w = workloads.make(args.config, n_trials=sample_trials)
    prob = w.oracle_problem()
    lookups = w.lookups()
    for _ in range(args.warmup):
        oracle.ylt(prob, want_gross=False)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        y, _, _ = oracle.ylt(prob, want_gross=False)
        oracle.metrics(y, w.probs)
    dt = (time.perf_counter() - t0) / args.steps
    value = lookups / dt
    cores = oracle.num_threads()
    sample = f"first {sample_trials} trials of workload {args.config} (all layers), YLT + metrics per step"
    line = {"impl": "reference", "metric": "trial-events x ELTs per second", "value": value,
            "unit": "trial-events*ELTs/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.config, "description": CONFIG_TEXT.get(args.config, ""),
                       "sample_trials": sample_trials},
            "cpu_baseline": {"value": value, "unit": "trial-events*ELTs/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "trial-events*ELTs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(args, w_full):
    """Oracle timed on the host cores on the first trials of the workload,
    as many as take about --cpu-seconds (all of them when they take less):
    the count is calibrated on 500 trials, then on about one second's worth
    (a small sample understates the threads' rate)."""
    import oracle
    T = w_full.yet.n_trials
    prob = w_full.oracle_problem()
    per_trial = w_full.lookups() / T

    def timed(n):
        t0 = time.perf_counter()
        oracle.ylt(prob, trials=np.arange(n, dtype=np.int64), want_gross=False)
        return time.perf_counter() - t0

    n = min(T, 500)
    dt = timed(n)
    for target in (1.0, args.cpu_seconds):
        n = int(min(T, max(n, target * n / max(dt, 1e-6))))
        dt = timed(n)
    return {"value": n * per_trial / dt, "unit": "trial-events*ELTs/s", "cores": oracle.num_threads(),
            "kind": "oracle", "sample": f"YLT of the first {n} of {T} trials, all layers ({dt:.1f} s)"}


def time_forward(art, torch, p, T, ids, off, K, ylt, stream, reps: int, warm: int = 1) -> float:
    """Mean forward ms over `reps` launches after `warm` untimed ones."""
    for _ in range(warm):
        art.art_run_ylt(p, T, ids, off, K, ylt, None, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        art.art_run_ylt(p, T, ids, off, K, ylt, None, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def link_probe(torch, src, dev, nbytes: int, reps: int = 8) -> dict:
    """The host-to-device link on its own: `reps` back-to-back copies of the
    host-run path's chunk size from the same pinned buffer, each timed with
    events; median and the whole run's rate."""
    n = min(src.numel(), nbytes // src.element_size())
    dst = torch.empty(n, dtype=src.dtype, device=dev)
    dst.copy_(src[:n], non_blocking=True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    ev[0].record()
    for i in range(reps):
        dst.copy_(src[:n], non_blocking=True)
        ev[i + 1].record()
    torch.cuda.synchronize(dev)
    each = [ev[i].elapsed_time(ev[i + 1]) for i in range(reps)]
    b = n * src.element_size()
    out = {"copy_bytes": b, "copies": reps, "median_gbs": b / (statistics.median(each) * 1e-3) / 1e9,
           "run_gbs": reps * b / (ev[0].elapsed_time(ev[reps]) * 1e-3) / 1e9}
    del dst
    return out


VMAP_NAMES = ("plain", "batched", "fp64", "skip", "sparse")


def extra_workload(name: str, dev, probes: dict, hbm: float, l2_size: float) -> dict:
    """One of the batching (c2), differentiation (c3) or precision (c4)
    workloads at full size, after the headline's timed region: forward time
    of each variant, the autotuned choice and its roofline; for c3 the whole
    step with the adjoint; for c4 the all-FP64 variant and the mixed
    variant's error against it."""
    import torch
    from paper_1308_2572_gb300 import art, workloads
    vmap = {"plain": art.ART_VARIANT_PLAIN, "batched": art.ART_VARIANT_BATCHED, "fp64": art.ART_VARIANT_FP64,
            "skip": art.ART_VARIANT_SKIP, "sparse": art.ART_VARIANT_SPARSE}
    t_gen = time.perf_counter()
    w = workloads.make(name)
    port, yet = w.portfolio, w.yet
    L, T, K = port.n_layers, yet.n_trials, yet.events_per_trial
    layouts = art.ART_LAYOUT_LAYER | art.ART_LAYOUT_POOL | art.ART_LAYOUT_SPARSE
    if name == "c3":
        layouts |= art.ART_LAYOUT_GROUP
    if name == "c4":
        layouts |= art.ART_LAYOUT_OCC64
    p = art.portfolio_from_workload(w, device=dev, layouts=layouts)
    ids = torch.from_numpy(yet.event_ids).to(dev)
    off = None if yet.trial_off is None else torch.from_numpy(yet.trial_off).to(dev)
    ylt = torch.empty((L, T), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    rec = {"description": CONFIG_TEXT.get(name, ""), "layers": L, "trials": T, "events": yet.n_events,
           "lookups_per_step": w.lookups(), "setup_s": round(time.perf_counter() - t_gen, 1)}
    try:
        fwd = {}
        for v in ("skip", "sparse", "batched", "plain"):
            art.art_set_variant(p, vmap[v])
            slow = v == "plain"
            fwd[v] = time_forward(art, torch, p, T, ids, off, K, ylt, stream, reps=1 if slow else 3)
        rec["forward_ms_by_variant_default_shapes"] = fwd
        tune = art.art_autotune(p, T, ids, off, K, ylt, sample_trials=min(T, 65536), stream=stream)
        inv = {v: k for k, v in vmap.items()}
        chosen = inv.get(tune["variant"], "skip")
        ms = time_forward(art, torch, p, T, ids, off, K, ylt, stream, reps=5)
        rec.update(variant=chosen, autotune=tune, forward_ms=ms, ms_per_1M_trial_ylt=ms * 1e6 / T,
                   trial_events_elts_per_s=w.lookups() / (ms * 1e-3),
                   vs_plain_one_layer_per_launch=fwd["plain"] / ms)
        ab = algorithmic_bytes(w, chosen, l2_size, builds_from_csr(port, layouts, chosen))
        roof = roofline(ab, ms * 1e-3, hbm, probes.get("l2_gather32_gbs"),
                        probes.get("fp64_add_gflops") if chosen == "fp64" else None)
        roof.update(kernel=VARIANT_KERNEL[chosen], traffic=recorded_traffic(VARIANT_KERNEL[chosen], name))
        rec["roofline"] = roof
        rec["lookups_performed_per_step"] = ab["lookups_performed"]
        probs = list(w.probs)
        n_p = len(probs)
        mean = torch.empty(L, dtype=torch.float64, device=dev)
        pml = torch.empty((L, n_p), dtype=torch.float64, device=dev)
        tvar = torch.empty((L, n_p), dtype=torch.float64, device=dev)
        art.art_run_ylt(p, T, ids, off, K, ylt, None, stream)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        for _ in range(5):
            art.art_metrics(ylt, T, L, probs, mean, pml, tvar, stream)
        e[1].record(stream)
        torch.cuda.synchronize(dev)
        rec["metrics_ms"] = e[0].elapsed_time(e[1]) / 5
        if name == "c3":
            art.art_set_variant(p, vmap[chosen])
            branch = torch.empty((L, T), dtype=torch.uint8, device=dev)
            gylt = torch.empty_like(ylt)
            ones_l = torch.ones(L, dtype=torch.float64, device=dev)
            ones_lp = torch.ones((L, n_p), dtype=torch.float64, device=dev)
            gterms = torch.empty((L, 4), dtype=torch.float64, device=dev)
            gmult = torch.empty(port.n_elt, dtype=torch.float64, device=dev)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            parts = {"forward": [], "metrics": [], "metrics_backward": [], "adjoint": []}
            for i in range(8):
                ev[0].record(stream)
                art.art_run_ylt(p, T, ids, off, K, ylt, branch, stream)
                ev[1].record(stream)
                art.art_metrics(ylt, T, L, probs, mean, pml, tvar, stream)
                ev[2].record(stream)
                art.art_metrics_backward(ylt, T, L, probs, pml, ones_l, ones_lp, gylt, stream)
                ev[3].record(stream)
                art.art_run_ylt_backward(p, T, ids, off, K, branch, gylt, gterms, gmult, stream)
                ev[4].record(stream)
                torch.cuda.synchronize(dev)
                if i >= 3:
                    for k, n in enumerate(parts):
                        parts[n].append(ev[k].elapsed_time(ev[k + 1]))
            rec["step_with_gradients_ms"] = float(np.mean([sum(x) for x in zip(*parts.values())]))
            rec["step_parts_ms"] = {k: float(np.mean(v)) for k, v in parts.items()}
            rec["gradients"] = "d(EL_j + TVaR_0.99,j)/d(OccR, OccL, AggR, AggL) per layer and d/d(m_e) per ELT"
        if name == "c4":
            # the all-FP64 variant and the mixed one's error against it (the
            # all-FP64 variant equals the FP64 oracle: tests/test_gpu_precision.py)
            art.art_set_variant(p, art.ART_VARIANT_FP64)
            y64 = torch.empty_like(ylt)
            rec["fp64_forward_ms"] = time_forward(art, torch, p, T, ids, off, K, y64, stream, reps=2)
            r64 = roofline(algorithmic_bytes(w, "fp64", l2_size, builds_from_csr(port, layouts, "fp64")),
                           rec["fp64_forward_ms"] * 1e-3, hbm,
                           probes.get("l2_gather32_gbs"), probes.get("fp64_add_gflops"))
            rec["fp64_roofline"] = {k: r64.get(k) for k in ("bound", "achieved", "peak", "unit", "frac", "t_star_ms",
                                                           "hbm_frac_by_dram_bytes", "peak_source")}
            art.art_set_variant(p, vmap[chosen])
            art.art_run_ylt(p, T, ids, off, K, ylt, None, stream)
            # the gross loss G per (layer, trial): the all-FP64 forward with
            # identity terms (no deductible, limit, retention or cap)
            m0, d0, l0, t0 = art.art_get_terms(p)
            ident = np.tile(np.array([0.0, np.inf, 0.0, np.inf]), (L, 1))
            gross = torch.empty_like(ylt)
            try:
                art.art_update_terms(p, elt_ded=np.zeros_like(d0), elt_lim=np.full_like(l0, np.inf), terms=ident)
                art.art_set_variant(p, art.ART_VARIANT_FP64)
                art.art_run_ylt(p, T, ids, off, K, gross, None, stream)
                torch.cuda.synchronize(dev)
            finally:
                art.art_update_terms(p, elt_mult=m0, elt_ded=d0, elt_lim=l0, terms=t0)
            rel = (ylt - y64).abs() / torch.where(gross > 0, gross, torch.ones_like(gross))
            m64, p64, t64 = (torch.empty_like(mean), torch.empty_like(pml), torch.empty_like(tvar))
            art.art_metrics(y64, T, L, probs, m64, p64, t64, stream)
            art.art_metrics(ylt, T, L, probs, mean, pml, tvar, stream)
            torch.cuda.synchronize(dev)
            relv = lambda a, b: torch.where(a == b, torch.zeros_like(a), (a - b).abs() / b.abs().clamp_min(1e-300))
            relerr = lambda a, b: float(relv(a, b).max())
            # the worst PML: its layer's aggregate over the PML bounds the
            # relative error that FP32 occurrence losses (relative rounding
            # 2^-24 each) can leave in Y = S - AggR
            rp = relv(pml, p64)
            wj, wq = divmod(int(torch.argmax(rp)), n_p)
            amp = (float(port.agg_ret[wj]) + float(p64[wj, wq])) / max(float(p64[wj, wq]), 1e-300)
            rec["precision_vs_all_fp64"] = {
                "trials": T, "max_abs_dy_over_gross": float(rel.max()),
                "pml_rel_err_by_prob": {str(pr): relerr(pml[:, q], p64[:, q]) for q, pr in enumerate(probs)},
                "tvar_rel_err_by_prob": {str(pr): relerr(tvar[:, q], t64[:, q]) for q, pr in enumerate(probs)},
                "mean_rel_err": relerr(mean, m64),
                "worst_pml": {"layer": wj, "prob": probs[wq], "pml": float(p64[wj, wq]),
                              "agg_ret": float(port.agg_ret[wj]), "aggregate_over_pml": amp,
                              "rel_err": float(rp[wj, wq]),
                              "rel_err_over_2^-24_x_aggregate_over_pml": float(rp[wj, wq]) / (amp * 2.0 ** -24)},
                "note": f"mixed ({chosen}) against the all-FP64 GPU variant on every (layer, trial)"}
            del y64, gross, rel
    finally:
        p.close()
        del ylt, ids, off
        torch.cuda.empty_cache()
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--config", default="c1")
    ap.add_argument("--variant", default="auto", choices=["auto", "plain", "batched", "fp64", "skip", "sparse"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=16)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-trials", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-probes", action="store_true", help="skip the libart bandwidth probes")
    ap.add_argument("--workloads", default="c2,c3,c4",
                    help="further workloads timed after the headline (comma list, or none)")
    ap.add_argument("--graph", action="store_true",
                    help="ART_FLAG_GRAPH: the forward's launches replay from a captured CUDA graph")
    ap.add_argument("--no-l2-persist", action="store_true",
                    help="no persisting L2 access-policy window over the gathered table (ART_FLAG_L2_PERSIST is "
                         "set by default: 5%% off the one-layer forward)")
    ap.add_argument("--trials", type=int, default=0,
                    help="keep only the first N trials (small cases for profiling; 0 = the full workload)")
    ap.add_argument("--layers", type=int, default=0,
                    help="keep only the first N layers (small cases for profiling; 0 = all)")
    ap.add_argument("--metrics-only", action="store_true",
                    help="time art_metrics alone on a synthetic YLT of --layers x --trials (128 x 1,000,000)")
    ap.add_argument("--probs", default="0.99,0.996,0.999", help="probabilities of --metrics-only")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.metrics_only:
        return run_metrics_only(args)

    import torch
    from paper_1308_2572_gb300 import art, shard, workloads

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    l2_size = float(torch.cuda.get_device_properties(dev).L2_cache_size)

    # the differentiation workload (c3) steps forward and backward; the
    # others, on more than one GPU, shard one YLT: each rank draws its own
    # YET of the workload's recipe (the same portfolio), and the metrics of
    # the whole YLT come from the ranks' top-k lists, all-gathered and merged
    with_grad = args.config == "c3"
    sharded = world > 1 and not with_grad
    t_gen = time.perf_counter()
    w = workloads.make(args.config, n_trials=args.trials or None, shard=rank if sharded else 0)
    if args.layers:
        w = first_layers(w, args.layers)
    log(f"[bench] rank {rank}: generated {args.config} in {time.perf_counter() - t_gen:.1f} s")
    port, yet = w.portfolio, w.yet
    L, T, K = port.n_layers, yet.n_trials, yet.events_per_trial
    # a named variant builds only the layouts it reads (keeps profiling runs
    # small); the skip variant's tables are built from the CSR
    layouts = {"plain": art.ART_LAYOUT_LAYER, "skip": art.ART_LAYOUT_LAYER | art.ART_LAYOUT_SPARSE,
               "batched": art.ART_LAYOUT_POOL,
               "fp64": art.ART_LAYOUT_LAYER | art.ART_LAYOUT_OCC64 | art.ART_LAYOUT_SPARSE,
               "sparse": art.ART_LAYOUT_SPARSE}.get(
        args.variant, art.ART_LAYOUT_LAYER | art.ART_LAYOUT_POOL | art.ART_LAYOUT_GROUP | art.ART_LAYOUT_SPARSE)
    if args.config == "c3":
        layouts |= art.ART_LAYOUT_GROUP  # the adjoint reads the group tables
    args.l2_persist = not args.no_l2_persist
    base_flags = (art.ART_FLAG_L2_PERSIST if args.l2_persist else 0) | (art.ART_FLAG_GRAPH if args.graph else 0)
    p = art.portfolio_from_workload(w, device=dev, layouts=layouts, flags=base_flags)
    ids = torch.from_numpy(yet.event_ids).to(dev)
    off = None if yet.trial_off is None else torch.from_numpy(yet.trial_off).to(dev)
    ylt = torch.empty((L, T), dtype=torch.float64, device=dev)
    probs = list(w.probs)
    n_p = len(probs)
    mean = torch.empty(L, dtype=torch.float64, device=dev)
    pml = torch.empty((L, n_p), dtype=torch.float64, device=dev)
    tvar = torch.empty((L, n_p), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    vmap = {"plain": art.ART_VARIANT_PLAIN, "batched": art.ART_VARIANT_BATCHED, "fp64": art.ART_VARIANT_FP64,
            "skip": art.ART_VARIANT_SKIP, "sparse": art.ART_VARIANT_SPARSE}

    # c3: branch codes in the forward, then dLoss/dYLT for sum(EL + TVaR)
    # and the adjoint
    branch = torch.empty((L, T), dtype=torch.uint8, device=dev) if with_grad else None
    gylt = torch.empty_like(ylt) if with_grad else None
    ones_l = torch.ones(L, dtype=torch.float64, device=dev)
    ones_lp = torch.ones((L, n_p), dtype=torch.float64, device=dev)
    gterms = torch.empty((L, 4), dtype=torch.float64, device=dev)
    gmult = torch.empty(port.n_elt, dtype=torch.float64, device=dev)

    def metrics():
        if sharded:
            shard.sharded_metrics(ylt, world * T, probs, stream=stream)
        else:
            art.art_metrics(ylt, T, L, probs, mean, pml, tvar, stream)

    def step():
        art.art_run_ylt(p, T, ids, off, K, ylt, branch, stream)
        metrics()
        if with_grad:
            art.art_metrics_backward(ylt, T, L, probs, pml, ones_l, ones_lp, gylt, stream)
            art.art_run_ylt_backward(p, T, ids, off, K, branch, gylt, gterms, gmult, stream)

    # variant choice: time each candidate forward (untimed for the result)
    cands = [args.variant] if args.variant != "auto" else ["plain", "batched", "skip", "sparse"]
    fwd_ms = {}
    for v in cands:
        art.art_set_variant(p, vmap[v])
        fwd_ms[v] = time_forward(art, torch, p, T, ids, off, K, ylt, stream, reps=3, warm=2)
    variant = min(fwd_ms, key=fwd_ms.get)
    tune = None
    if args.variant == "auto":
        # the library's autotuner picks the variant and tile shapes on a sample
        tune = art.art_autotune(p, T, ids, off, K, ylt, sample_trials=min(T, 65536), stream=stream)
        inv = {v: k for k, v in vmap.items()}
        variant = inv.get(tune["variant"], variant)
    else:
        art.art_set_variant(p, vmap[variant])
    log(f"[bench] forward ms per variant (default shapes): {fwd_ms}; using {variant} {tune or ''}")

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    assert art.art_get_device_status(p, stream) == art.ART_OK

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    start.record(stream)
    for i in range(args.steps):
        ev[i][0].record(stream)
        art.art_run_ylt(p, T, ids, off, K, ylt, branch, stream)
        ev[i][1].record(stream)
        metrics()
        if with_grad:
            art.art_metrics_backward(ylt, T, L, probs, pml, ones_l, ones_lp, gylt, stream)
            art.art_run_ylt_backward(p, T, ids, off, K, branch, gylt, gterms, gmult, stream)
    end.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    total_ms = start.elapsed_time(end)
    fwd = [a.elapsed_time(b) for a, b in ev]
    total_ms = rank_max(total_ms, dist, dev)
    if dist:
        dist.barrier()
    ms_step = total_ms / args.steps
    lookups = w.lookups()
    value = whole_job_rate(lookups * args.steps, world, total_ms / 1e3)
    fwd_mean = float(np.mean(fwd))

    # measured limits the copy-bandwidth and GEMM peaks do not cover (libart probes)
    probes = {}
    if rank == 0 and not args.no_probes:
        probes = {"l2_gather32_gbs": art.art_probe(art.ART_PROBE_GATHER32, 64 << 20),
                  "l2_gather64_gbs": art.art_probe(art.ART_PROBE_GATHER64, 64 << 20),
                  "dram_gather32_gbs": art.art_probe(art.ART_PROBE_GATHER32, 8 << 30, 3),
                  "stream_read_gbs": art.art_probe(art.ART_PROBE_STREAM, 8 << 30, 3),
                  "fp64_add_gflops": art.art_probe(art.ART_PROBE_FP64ADD, 0, 3)}
    # roofline of the dominant kernel (the forward)
    peak, peak_kind = measured_peaks()
    ab = algorithmic_bytes(w, variant, l2_size, builds_from_csr(port, layouts, variant))
    roof = roofline(ab, fwd_mean / 1e3, peak, probes.get("l2_gather32_gbs"),
                    probes.get("fp64_add_gflops") if variant == "fp64" else None)
    kernel_name = VARIANT_KERNEL[variant]
    roof.update(kernel=kernel_name, traffic=recorded_traffic(kernel_name, args.config),
                hbm_peak_source=f"{peak_kind} hbm_gbs {peak} GB/s (copy bandwidth)")
    if probes:
        roof["probes"] = probes

    # end to end through the C ABI with host buffers: the pinned YET goes to
    # the device in chunks, the forward and the metrics run there, the YLT
    # and the metrics come back
    e2e = None
    if args.e2e_steps > 0:
        ids_h = torch.from_numpy(yet.event_ids).pin_memory()
        assert ids_h.is_pinned()
        off_h = None if yet.trial_off is None else torch.from_numpy(yet.trial_off).pin_memory()
        ylt_h = torch.empty((L, T), dtype=torch.float64).pin_memory()
        mean_h = torch.empty(L, dtype=torch.float64).pin_memory()
        pml_h = torch.empty((L, n_p), dtype=torch.float64).pin_memory()
        tvar_h = torch.empty((L, n_p), dtype=torch.float64).pin_memory()

        def e2e_step():
            if sharded:
                # the shard's YLT comes back to the host and goes to the
                # device again for the top-k lists: the host-buffer call
                # returns the YLT, and the merge needs every rank's lists
                art.art_run_ylt_host(p, T, ids_h, off_h, K, ylt_h, stream)
                ylt.copy_(ylt_h, non_blocking=True)
                shard.sharded_metrics(ylt, world * T, probs, stream=stream)
            else:
                art.art_run_ylt_host_metrics(p, T, ids_h, off_h, K, probs, ylt=ylt_h, mean=mean_h, pml=pml_h,
                                             tvar=tvar_h, stream=stream)

        for _ in range(args.warmup):  # the first calls grow the staging, YLT and scratch buffers
            e2e_step()
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        each = []
        for _ in range(args.e2e_steps):
            t1 = time.perf_counter()
            e2e_step()  # blocks until the results are in host memory
            each.append((time.perf_counter() - t1) * 1e3)
        e2e_s = rank_max((time.perf_counter() - t0) / args.e2e_steps, dist, dev)
        # the bytes the step moves: the YET (and offsets) in, the YLT and the metrics out
        h2d = yet.event_ids.nbytes + (0 if yet.trial_off is None else yet.trial_off.nbytes)
        d2h = 8 * L * T + 8 * L * (1 + 2 * n_p)
        if sharded:
            h2d += 8 * L * T  # the shard's YLT back to the device
            d2h = 8 * L * T + 8 * L * (shard.list_length(world * T, probs) * world + world)
        link = link_probe(torch, ids_h, dev, 64 << 20)
        e2e = {"value": whole_job_rate(lookups, world, e2e_s), "unit": "trial-events*ELTs/s",
               "ms_per_step": e2e_s * 1e3, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_each_step_rank0": [round(t, 3) for t in each],
               "step_h2d_gbs": h2d / e2e_s / 1e9, "h2d_link_rank0": link,
               "path": ("art_run_ylt_host per rank, the shard's YLT to the device, art_topk, all-gather, host "
                        "merge (art_merge_topk)") if sharded else
                       ("art_run_ylt_host_metrics (the pinned host YET read in place over the host link by a "
                        "forward that reads every id once, else copied in 64 MiB chunks overlapped with the "
                        "forward; YLT kept on the device for art_metrics; YLT and metrics copied back)")}
        del ids_h, ylt_h

    # optional early exit (capped trials stop being read), reported separately
    early = None
    if variant == "skip":
        art.art_set_flags(p, art.ART_FLAG_EARLY_EXIT | base_flags)
        early = {"forward_ms": time_forward(art, torch, p, T, ids, off, K, ylt, stream, reps=5),
                 "note": "ART_FLAG_EARLY_EXIT: trials stop being read once capped; not part of value"}
        art.art_set_flags(p, base_flags)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args, w)

    # kernels of ours launched per step: forward (one per layer for the plain
    # variant; one occurrence-table build plus a trial pass per occurrence
    # group for the skip and all-FP64 variants; one persistent launch
    # otherwise) + metrics (6 radix passes, each fused with its digit pick,
    # and the tail sums fused with the final reduction)
    n_groups = len(layer_groups(port))
    launches = {"plain": L, "skip": 1 + len(occurrence_groups(port)),
                "fp64": 1 + len(occurrence_groups(port, 4))}.get(variant, 1) + 7
    if with_grad:
        # metrics backward (count, weights, grad) + the adjoint: per group the
        # event masks, a pass and its reduction (group tables), else per layer
        # a pass and its reduction plus one scatter
        launches += 3 + (3 * n_groups if layouts & art.ART_LAYOUT_GROUP else 2 * L + 1)
    config = {"workload": args.config, "description": CONFIG_TEXT.get(args.config, ""),
              "variant": variant, "autotune": tune, "l2_persist": bool(args.l2_persist), "graph": bool(args.graph),
              "layers": L, "trials": T, "events": yet.n_events,
              "lookups_per_step": lookups, "lookups_performed_per_step": ab["lookups_performed"],
              "l2": "inputs larger than L2 (the 4 GB YET is re-streamed every step)",
              "parallelism": (f"{world} ranks sharding one YLT of {world} x {T} trials: each rank its own YET "
                              "shard; per-layer top-k lists and sums all-gathered (NCCL) and merged exactly for "
                              "the metrics (weak scaling)") if sharded else
                             (f"{world} independent ranks (weak scaling, no collective in the data path)"
                              if world > 1 else "one GPU")}
    p.close()
    del ylt, ids, off
    torch.cuda.empty_cache()

    extras = {}
    names = [] if args.workloads in ("", "none") else [n for n in args.workloads.split(",") if n != args.config]
    # the other workloads are single-GPU figures: timed at N = 1 only, so that
    # the ranks of a scaling run are not held while rank 0 times them
    if rank == 0 and world == 1 and not args.trials and not args.layers:
        for name in names:
            t0 = time.perf_counter()
            try:
                extras[name] = extra_workload(name, dev, probes, peak, l2_size)
            except Exception as ex:  # reported, not fatal: the headline stands on its own
                extras[name] = {"error": f"{type(ex).__name__}: {ex}"}
            extras[name]["wall_s"] = round(time.perf_counter() - t0, 1)
            log(f"[bench] {name}: {json.dumps(extras[name])[:400]}")
    if dist:
        dist.barrier()

    if rank == 0:
        line = {
            "metric": "trial-events x ELTs per second", "value": value, "unit": "trial-events*ELTs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic", "config": config,
            "ms_per_1M_trial_ylt": fwd_mean * 1e6 / T,
            "forward_ms": fwd_mean, "forward_ms_by_variant": fwd_ms,
            "roofline": roof, "clocks": clk, "e2e": e2e, "early_exit": early, "gpu_launches": launches * args.steps,
            "cpu_baseline": cpu, "workloads": extras or None,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())

"""Precision report for the 128-layer, 512-ELT workload (mixed vs all-FP64).

Runs every forward variant (the all-FP64 one over FP64 occurrence tables
and over the FP64 pool) through the C ABI on the first N trials of the
precision workload (lognormal(13, 2.5) pool, 1,000 events per trial), and
the FP64 oracle on the same trials, then reports per variant:
  - max over (layer, trial) of |dY| / G (G = the trial's gross loss; the
    tolerance is 1e-6),
  - max relative error of PML and TVaR at p = 0.99, 0.996, 0.999 (GPU metrics
    of the GPU YLT against the oracle's metrics of the oracle's YLT; the
    tolerance is 1e-6),
  - the forward time on those trials.

    python tests/precision_report.py [--trials 20000] [--config c4]

Prints one JSON object. Test infrastructure: it calls the oracle.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1308_2572_gb300 import art, workloads  # noqa: E402

MIXED = (1 | 2 | 8 | 16)  # layer, pool, group and CSR layouts (ART_LAYOUT_*)
VARIANTS = {"batched (FP32 + FP64 aggregate)": ("ART_VARIANT_BATCHED", MIXED), "sparse": ("ART_VARIANT_SPARSE", MIXED),
            "skip": ("ART_VARIANT_SKIP", MIXED), "plain": ("ART_VARIANT_PLAIN", MIXED),
            "all-FP64 (occurrence tables)": ("ART_VARIANT_FP64", 1 | 16 | 32),
            "all-FP64 (FP64 pool)": ("ART_VARIANT_FP64", 4)}


def report(config: str = "c4", n_trials: int = 20000) -> dict:
    import torch
    w = workloads.make(config, n_trials=n_trials)
    probs = [0.99, 0.996, 0.999]
    t0 = time.perf_counter()
    ref, gross, _ = oracle.ylt(w.oracle_problem())
    t_oracle = time.perf_counter() - t0
    om, op, ot = oracle.metrics(ref, probs)
    ids = torch.from_numpy(w.yet.event_ids).cuda()
    off = None if w.yet.trial_off is None else torch.from_numpy(w.yet.trial_off).cuda()
    L, T, K = w.portfolio.n_layers, w.yet.n_trials, w.yet.events_per_trial
    out = {"config": config, "trials": T, "layers": L, "probs": probs, "oracle_seconds": t_oracle,
           "oracle_threads": oracle.num_threads(), "variants": {}}
    for name, (v, layouts) in VARIANTS.items():
        p = art.portfolio_from_workload(w, layouts=layouts)
        art.art_set_variant(p, getattr(art, v))
        ylt = torch.empty((L, T), dtype=torch.float64, device="cuda")
        art.art_run_ylt(p, T, ids, off, K, ylt)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        art.art_run_ylt(p, T, ids, off, K, ylt)
        e1.record()
        torch.cuda.synchronize()
        y = ylt.cpu().numpy()
        with np.errstate(divide="ignore", invalid="ignore"):
            rel = np.where(gross > 0, np.abs(y - ref) / np.where(gross > 0, gross, 1), np.abs(y - ref))
        mean = torch.empty(L, dtype=torch.float64, device="cuda")
        pml = torch.empty((L, 3), dtype=torch.float64, device="cuda")
        tvar = torch.empty((L, 3), dtype=torch.float64, device="cuda")
        art.art_metrics(ylt, T, L, probs, mean, pml, tvar)
        pml, tvar, mean = pml.cpu().numpy(), tvar.cpu().numpy(), mean.cpu().numpy()
        relerr = lambda a, b: float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))
        out["variants"][name] = {
            "max_abs_dY_over_G": float(rel.max()),
            "max_rel_dY_where_Y_positive": float(np.max(np.where(ref > 0, np.abs(y - ref) / np.where(ref > 0, ref, 1), 0))),
            "pml_rel_err": [relerr(pml[:, q], op[:, q]) for q in range(3)],
            "tvar_rel_err": [relerr(tvar[:, q], ot[:, q]) for q in range(3)],
            "mean_rel_err": relerr(mean, om),
            "forward_ms": e0.elapsed_time(e1),
        }
        p.close()
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="c4")
    ap.add_argument("--trials", type=int, default=20000)
    a = ap.parse_args()
    print(json.dumps(report(a.config, a.trials), indent=1))

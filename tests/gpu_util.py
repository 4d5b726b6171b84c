"""Shared helpers for the GPU parity tests (CUDA path vs FP64 oracle)."""
import numpy as np
import torch

import oracle
from paper_1308_2572_gb300 import art

# Spec tolerances: |dY| <= 1e-6 x (trial's gross loss) per (trial,
# layer); PML and TVaR within 1e-6 relative.
YLT_TOL = 1e-6
METRIC_RTOL = 1e-6


def device_yet(w, device="cuda"):
    ids = torch.from_numpy(w.yet.event_ids).to(device)
    off = None if w.yet.trial_off is None else torch.from_numpy(w.yet.trial_off).to(device)
    return ids, off, w.yet.events_per_trial, w.yet.n_trials


def run_ylt(p, w, variant, yet=None, branch=False, device="cuda"):
    ids, off, k, T = yet if yet is not None else device_yet(w, device)
    art.art_set_variant(p, variant)
    L = w.portfolio.n_layers
    ylt = torch.full((L, T), -1.0, dtype=torch.float64, device=device)
    br = torch.full((L, T), 255, dtype=torch.uint8, device=device) if branch else None
    art.art_run_ylt(p, T, ids, off, k, ylt, br)
    torch.cuda.synchronize()
    assert art.art_get_device_status(p) == art.ART_OK
    return ylt, br


def assert_ylt_close(gpu, ref, gross, what=""):
    """|dY| <= 1e-6 G element by element; returns the max of |dY| / G."""
    gpu = np.asarray(gpu)
    err = np.abs(gpu - ref)
    bad = err > YLT_TOL * gross
    if np.any(bad):
        j, t = np.argwhere(bad)[0]
        raise AssertionError(f"{what}: {int(bad.sum())} outputs off; first (layer {j}, trial {t}): "
                             f"gpu {gpu[j, t]!r} oracle {ref[j, t]!r} gross {gross[j, t]!r}")
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = np.where(gross > 0, err / np.where(gross > 0, gross, 1), 0.0)
    return float(rel.max()) if rel.size else 0.0


def gpu_metrics(ylt, probs):
    L, T = ylt.shape
    n_p = len(probs)
    mean = torch.empty(L, dtype=torch.float64, device=ylt.device)
    pml = torch.empty((L, n_p), dtype=torch.float64, device=ylt.device)
    tvar = torch.empty((L, n_p), dtype=torch.float64, device=ylt.device)
    art.art_metrics(ylt, T, L, probs, mean, pml, tvar)
    torch.cuda.synchronize()
    return mean.cpu().numpy(), pml.cpu().numpy(), tvar.cpu().numpy()


def oracle_sample(w, trials):
    return oracle.ylt(w.oracle_problem(), trials=np.asarray(trials, dtype=np.int64))

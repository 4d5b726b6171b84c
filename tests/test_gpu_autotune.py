"""The autotuner: it times variants and tile shapes on a sample, keeps the
fastest, the result still matches the oracle, and a cache file replays it."""
import numpy as np
import pytest
import torch

import oracle
from paper_1308_2572_gb300 import art, workloads

from gpu_util import assert_ylt_close, device_yet

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_valid_shape_and_keeps_parity(tmp_path, monkeypatch):
    monkeypatch.setenv("ART_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    w = workloads.random_case(301, catalogue=4001, n_elt=60, n_layers=90, n_trials=6000, max_len=120,
                              max_elts_per_layer=32, nnz_frac=0.05)
    p = art.portfolio_from_workload(w)
    try:
        ids, off, k, T = device_yet(w)
        L = w.portfolio.n_layers
        ylt = torch.empty((L, T), dtype=torch.float64, device="cuda")
        r = art.art_autotune(p, T, ids, off, k, ylt, sample_trials=4000)
        assert r["from_cache"] == 0 and r["candidates"] > 10 and r["sample_ms"] > 0
        assert r["variant"] in (art.ART_VARIANT_PLAIN, art.ART_VARIANT_SKIP, art.ART_VARIANT_BATCHED,
                                art.ART_VARIANT_SPARSE)
        if r["variant"] in (art.ART_VARIANT_BATCHED, art.ART_VARIANT_SPARSE):
            assert r["slots"] in (2, 4, 8) and r["trial_tile"] in (1, 2, 4, 8, 16) and r["cta_threads"] in (128, 256)
        art.art_run_ylt(p, T, ids, off, k, ylt)
        torch.cuda.synchronize()
        ref, gross, _ = oracle.ylt(w.oracle_problem())
        assert_ylt_close(ylt.cpu().numpy(), ref, gross, "autotuned")
        r2 = art.art_autotune(p, T, ids, off, k, ylt, sample_trials=4000)
        assert r2["from_cache"] == 1
        assert (r2["variant"], r2["slots"], r2["trial_tile"], r2["cta_threads"]) == \
               (r["variant"], r["slots"], r["trial_tile"], r["cta_threads"])
        assert (tmp_path / "tune.txt").read_text().count("\t") >= 2
    finally:
        p.close()


@pytest.mark.parametrize("slots_variant", ["batched", "sparse"])
def test_every_layer_tile_matches_the_oracle(tmp_path, monkeypatch, slots_variant):
    """Force each layer tile through the cache file (slots 2, 4, 8) and check
    parity: 90 layers need 2, 1 or 1 tiles of 64, 128, 256 layers."""
    w = workloads.random_case(302, catalogue=3001, n_elt=50, n_layers=90, n_trials=700, max_len=80,
                              max_elts_per_layer=32, nnz_frac=0.08)
    ref, gross, _ = oracle.ylt(w.oracle_problem())
    v = {"batched": art.ART_VARIANT_BATCHED, "sparse": art.ART_VARIANT_SPARSE}[slots_variant]
    shapes = [(slots, m) for slots in (2, 4, 8) for m in ((0, 1) if slots_variant == "sparse" else (-1,))]
    for slots, mapping in shapes:
        cache = tmp_path / f"tune_{slots}_{mapping}.txt"
        monkeypatch.setenv("ART_AUTOTUNE_CACHE", str(cache))
        p = art.portfolio_from_workload(w)
        try:
            ids, off, k, T = device_yet(w)
            L = w.portfolio.n_layers
            ylt = torch.empty((L, T), dtype=torch.float64, device="cuda")
            r = art.art_autotune(p, T, ids, off, k, ylt, sample_trials=200)
            # rewrite the recorded shape with the forced tile and replay it
            key = cache.read_text().splitlines()[-1].split("\t")[0]
            cache.write_text(f"{key}\t{v} {slots} 2 128 {mapping}\t0.0\n")
            r = art.art_autotune(p, T, ids, off, k, ylt, sample_trials=200)
            assert r["from_cache"] == 1 and r["slots"] == slots and r["variant"] == v and r["mapping"] == mapping
            ylt.fill_(-1.0)
            art.art_run_ylt(p, T, ids, off, k, ylt)
            torch.cuda.synchronize()
            assert art.art_get_device_status(p) == art.ART_OK
            assert_ylt_close(ylt.cpu().numpy(), ref, gross, f"{slots_variant} slots {slots} mapping {mapping}")
        finally:
            p.close()

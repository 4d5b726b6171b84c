"""bench.py's roofline bookkeeping (no GPU): the grouping it assumes matches
the library's rules, and each variant is accounted against the right
bound."""
import json
import types
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1308_2572_gb300 import workloads  # noqa: E402


def test_occurrence_groups_are_runs_of_consecutive_layers():
    w = workloads.random_case(901, n_elt=12, n_layers=19, n_trials=5)
    g8 = bench.occurrence_groups(w.portfolio)
    g4 = bench.occurrence_groups(w.portfolio, 4)
    assert [len(g) for g in g8] == [8, 8, 3] and [len(g) for g in g4] == [4, 4, 4, 4, 3]
    assert sum(g8, []) == list(range(19)) == sum(g4, [])


def test_layer_groups_respect_the_layer_and_elt_caps():
    w = workloads.random_case(902, n_elt=60, n_layers=40, n_trials=5, max_elts_per_layer=12)
    port = w.portfolio
    groups = bench.layer_groups(port, with_layers=True)
    assert sum((lays for _, lays in groups), []) == list(range(port.n_layers))
    for elts, lays in groups:
        assert 1 <= len(lays) <= 8 and len(elts) <= 32
        want = []
        for j in lays:
            for e in port.layer_elt_ids[port.layer_elt_off[j]:port.layer_elt_off[j + 1]]:
                if int(e) not in want:
                    want.append(int(e))
        assert elts == want  # union in order of first appearance


def test_occurrence_density_against_a_direct_count():
    w = workloads.make("c0u")
    port = w.portfolio
    x = np.zeros(port.catalogue_size)
    for e in port.layer_elt_ids[port.layer_elt_off[0]:port.layer_elt_off[1]]:
        l = port.elt_losses[e].astype(np.float64)
        x += np.clip(float(port.elt_mult[e]) * l - float(port.elt_ded[e]), 0.0, float(port.elt_lim[e]))
    want = float(np.mean(x > float(port.occ_ret[0])))
    assert bench.occurrence_density(port, [0]) == want
    assert 0.0 < want < 1.0


def test_each_variant_is_accounted_against_its_bound():
    w = workloads.make("c0", n_trials=200)
    for v in ("plain", "skip", "batched", "sparse"):
        ab = bench.algorithmic_bytes(w, v)
        assert {"s8d", "compulsory", "l2", "table_bytes", "l2_resident", "lookups_performed"} <= set(ab), v
        assert ab["s8d"] >= ab["compulsory"] > 0
    ab = bench.algorithmic_bytes(w, "fp64")
    # the all-FP64 variant's FP64 operations are its build's: an FMA per
    # non-zero loss and an add per (loss, layer holding it)
    port = w.portfolio
    nnz = float((port.elt_losses != 0).sum())
    assert ab["fp64_flops"] == pytest.approx(2 * nnz + nnz * float(port.elts_per_layer().sum()) / port.n_elt)


def test_skip_variant_counts_the_lookups_it_performs():
    """The memoised forward reads each catalogue event's row once per layer
    ELT in its build and one row of X per event with an occurrence loss."""
    w = workloads.make("c0u", n_trials=300)
    port = w.portfolio
    ab = bench.algorithmic_bytes(w, "skip")
    dens = bench.occurrence_density(port, [0])
    want = port.catalogue_size * int(port.elts_per_layer().sum()) + w.yet.n_events * dens
    assert ab["lookups_performed"] == want
    assert ab["lookups_performed"] < w.lookups()  # fewer than one per (occurrence, ELT)
    assert ab["table_bytes"] == 4 * (port.catalogue_size + 1) and ab["l2_resident"]
    plain = bench.algorithmic_bytes(w, "plain")
    assert plain["lookups_performed"] == w.lookups()


def test_roofline_of_an_l2_resident_table():
    """The one-layer paper-scale step as measured: 4.14 GB compulsory DRAM
    bytes, 7.01 GB of L2 sectors, 1.331 ms; HBM 6769.4 GB/s, probed L2 gather
    6956 GB/s. t* = max(0.612, 1.008) ms: L2-bound at 0.757, and 0.46 of HBM
    by the DRAM bytes alone."""
    ab = {"s8d": 7.02e9, "compulsory": 4.14e9, "l2": 7.01e9, "table_bytes": 8e6, "l2_resident": True}
    r = bench.roofline(ab, 1.331e-3, 6769.4, 6956.0)
    assert r["bound"] == "l2" and r["unit"] == "GB/s" and r["peak"] == 6956.0
    assert r["t_star_ms"] == pytest.approx(max(4.14e9 / 6769.4e9, 7.01e9 / 6956e9) * 1e3)
    assert r["frac"] == pytest.approx(r["t_star_ms"] / 1.331, rel=1e-12)
    assert r["frac"] == pytest.approx(0.757, abs=1e-3)
    assert r["hbm_frac_by_dram_bytes"] == pytest.approx(0.4595, abs=1e-3)
    assert r["achieved"] / r["peak"] == r["frac"]
    # a faster DRAM-side case flips the bound to HBM (compulsory bytes)
    r2 = bench.roofline(dict(ab, l2=1e9), 1.0e-3, 6769.4, 6956.0)
    assert r2["bound"] == "hbm" and r2["frac"] == pytest.approx(4.14e9 / 1e-3 / 6769.4e9)
    # no L2 probe: the DRAM term alone
    assert bench.roofline(ab, 1.331e-3, 6769.4, None)["bound"] == "hbm"


def test_roofline_of_a_table_larger_than_l2_and_of_fp64():
    ab = {"s8d": 68e9, "compulsory": 4.2e9, "l2": 68e9, "table_bytes": 128e6, "l2_resident": False}
    r = bench.roofline(ab, 11.2e-3, 6769.4, 6956.0)
    assert r["bound"] == "hbm" and r["frac"] == pytest.approx(68e9 / 11.2e-3 / 6769.4e9)
    # FP64 work that takes longer than the traffic names the bound ...
    r = bench.roofline(dict(ab, fp64_flops=1e11), 0.69, 6769.4, 6956.0, fp64_gflops=528.0)
    assert r["bound"] == "alu" and r["unit"] == "GFLOP/s" and r["frac"] == pytest.approx(1e11 / 0.69 / 528e9)
    assert r["t_star_ms"] == pytest.approx(1e11 / 528e9 * 1e3)
    # ... and FP64 work that takes less does not
    r = bench.roofline(dict(ab, fp64_flops=1e9), 11.2e-3, 6769.4, 6956.0, fp64_gflops=528.0)
    assert r["bound"] == "hbm" and r["frac"] == pytest.approx(68e9 / 11.2e-3 / 6769.4e9)
    res = dict(ab, l2_resident=True, compulsory=4.14e9, l2=7.01e9)
    r = bench.roofline(dict(res, fp64_flops=1e8), 1.331e-3, 6769.4, 6956.0, fp64_gflops=528.0)
    assert r["bound"] == "l2" and r["frac"] == pytest.approx(7.01e9 / 6956e9 / 1.331e-3)


def test_traffic_comes_from_a_json_record_of_the_current_sources(tmp_path):
    rec = {"kernel": "ylt_skip", "workload": "c1", "source_hash": bench.kernel_source_hash("ylt_skip"),
           "dram_bytes_per_launch": 4.06e9}
    (tmp_path / "ylt_skip_c1.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("ylt_skip", "c1", str(tmp_path)) == 4.06e9
    (tmp_path / "ylt_skip_c1.json").write_text(json.dumps(dict(rec, source_hash="0" * 16)))
    assert bench.recorded_traffic("ylt_skip", "c1", str(tmp_path)) is None  # stale sources
    assert bench.recorded_traffic("ylt_plain", "c1", str(tmp_path)) is None  # no record


def test_first_layers_keeps_a_consistent_prefix_of_the_portfolio():
    w = workloads.make("c0u", n_trials=20)
    big = workloads.random_case(903, n_elt=12, n_layers=9, n_trials=5)
    sub = bench.first_layers(big, 4).portfolio
    port = big.portfolio
    assert sub.n_layers == 4 and sub.layer_elt_off[-1] == sub.layer_elt_ids.size
    assert np.array_equal(sub.layer_elt_ids, port.layer_elt_ids[:port.layer_elt_off[4]])
    assert np.array_equal(sub.agg_lim, port.agg_lim[:4]) and sub.elt_losses is port.elt_losses
    assert bench.first_layers(w, 5).portfolio.n_layers == 1  # at most the layers there are


def test_csr_build_accounting():
    """With ART_LAYOUT_SPARSE the skip and all-FP64 builds read the CSR (per
    group: the offsets and every 8-byte entry) instead of the per-layer
    tables, whatever the order the layers list their ELTs in."""
    from paper_1308_2572_gb300 import art
    w = workloads.make("c0", n_trials=200)
    port = w.portfolio
    sparse = art.ART_LAYOUT_LAYER | art.ART_LAYOUT_SPARSE
    assert bench.csr_build_used(port, sparse)
    assert not bench.csr_build_used(port, art.ART_LAYOUT_LAYER)
    assert bench.builds_from_csr(port, sparse, "fp64") and not bench.builds_from_csr(port, sparse, "plain")
    dense = bench.algorithmic_bytes(w, "skip")
    csr = bench.algorithmic_bytes(w, "skip", csr_build=True)
    C = port.catalogue_size
    nnz = float((port.elt_losses != 0).sum())
    x_and_bits = (C + 1) * 4 + C / 8  # one layer: LP = 1, 4-byte entries
    assert csr["compulsory"] - (dense["compulsory"] - (4 * 4 * C + x_and_bits)) == pytest.approx(
        4.0 * (C + 1) + 8.0 * nnz + x_and_bits)
    assert csr["lookups_performed"] - dense["lookups_performed"] == pytest.approx(nnz - C * 3)
    rev = types.SimpleNamespace(**{k: getattr(port, k) for k in ("n_layers", "layer_elt_off")})
    ids = port.layer_elt_ids.copy()
    ids[port.layer_elt_off[0]:port.layer_elt_off[1]] = ids[port.layer_elt_off[0]:port.layer_elt_off[1]][::-1]
    rev.layer_elt_ids = ids
    assert bench.csr_build_used(rev, sparse)


def test_bench_help_renders():
    """Every help string of bench.py formats (argparse expands % in them)."""
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                                     "bench.py"), "--help"], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr[-500:]
    assert "--no-l2-persist" in r.stdout

"""bench.py's roofline bookkeeping (no GPU): the grouping it assumes matches
the library's rules, and each variant is accounted against the right
bound."""
import os
import sys

import numpy as np

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
        assert set(ab) == {"s8d", "compulsory", "l2"}, v
        assert ab["s8d"] >= ab["compulsory"] > 0
    ab = bench.algorithmic_bytes(w, "fp64")
    assert ab["fp64_flops"] > 0  # the all-FP64 variant is bound by the FP64 pipe

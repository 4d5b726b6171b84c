"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Small workloads are compared element by element in full; the paper-scale
workloads run in the launch configuration the bench times and are compared
on sampled trials the oracle computes one by one. Tolerance: |dY| <= 1e-6 x
the trial's gross loss for every (layer, trial).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1308_2572_gb300 import art, workloads

from gpu_util import assert_ylt_close, device_yet, gpu_metrics, oracle_sample, run_ylt, METRIC_RTOL

pytestmark = pytest.mark.gpu

VARIANTS = [art.ART_VARIANT_PLAIN, art.ART_VARIANT_BATCHED, art.ART_VARIANT_FP64, art.ART_VARIANT_SKIP,
            art.ART_VARIANT_SPARSE]
ALL_LAYOUTS = (art.ART_LAYOUT_LAYER | art.ART_LAYOUT_POOL | art.ART_LAYOUT_POOL64 | art.ART_LAYOUT_GROUP
               | art.ART_LAYOUT_SPARSE)
# the all-FP64 variant over FP64 occurrence tables (without them it runs over
# the FP64 pool, as in ALL_LAYOUTS)
OCC64_LAYOUTS = art.ART_LAYOUT_LAYER | art.ART_LAYOUT_OCC64
FP64_TOL = 1e-12  # |dY| <= 1e-12 G: FP64 arithmetic, only the summation order differs from the oracle


def _check_fp64_occ(w, ref, gross, what, trials=None):
    # tables built from the layer tables, and from the CSR of the non-zero losses
    for layouts in (OCC64_LAYOUTS, OCC64_LAYOUTS | art.ART_LAYOUT_SPARSE):
        p = art.portfolio_from_workload(w, layouts=layouts)
        try:
            ylt, _ = run_ylt(p, w, art.ART_VARIANT_FP64)
            y = ylt.cpu().numpy() if trials is None else ylt[:, torch.from_numpy(trials).cuda()].cpu().numpy()
            err = np.abs(y - ref)
            assert np.all(err <= FP64_TOL * np.maximum(gross, 1.0)), \
                f"{what}: FP64 occurrence tables (layouts {layouts}), max {err.max()}"
        finally:
            p.close()


def _small_cases():
    return {
        "ragged_csr_with_empty_trials": dict(seed=101, n_trials=1000, min_len=0, max_len=130),
        "dense_k37": dict(seed=102, n_trials=777, dense_k=37),
        "dense_k1": dict(seed=103, n_trials=300, dense_k=1),
        "single_trial": dict(seed=104, n_trials=1, min_len=250, max_len=250),
        "inf_limits": dict(seed=105, n_trials=500, inf_limits=True),
        "one_elt_layers": dict(seed=106, n_elt=9, n_layers=7, max_elts_per_layer=1, n_trials=400),
        "thirty_two_elt_layers": dict(seed=107, catalogue=1001, n_elt=40, n_layers=5, n_trials=300,
                                      max_elts_per_layer=32),
        "many_layers_two_tiles": dict(seed=108, catalogue=333, n_elt=70, n_layers=300, n_trials=200, max_len=40,
                                      max_elts_per_layer=32),
        "multipliers": dict(seed=109, n_trials=400, mult_range=(0.3, 2.5)),
        "wide_pool": dict(seed=110, catalogue=5003, n_elt=300, n_layers=20, n_trials=150, max_len=60,
                          max_elts_per_layer=32, nnz_frac=0.05),
    }


@pytest.mark.parametrize("case", sorted(_small_cases()))
def test_small_cases_all_variants(case):
    kw = _small_cases()[case]
    w = workloads.random_case(**kw)
    ref, gross, _ = oracle.ylt(w.oracle_problem())
    p = art.portfolio_from_workload(w, layouts=ALL_LAYOUTS)
    try:
        yet = device_yet(w)
        for v in VARIANTS:
            ylt, _ = run_ylt(p, w, v, yet=yet)
            assert_ylt_close(ylt.cpu().numpy(), ref, gross, f"{case} variant {v}")
    finally:
        p.close()
    _check_fp64_occ(w, ref, gross, case)


@pytest.mark.parametrize("name", ["c0", "c0u"])
def test_config0_full(name):
    w = workloads.make(name)
    ref, gross, _ = oracle.ylt(w.oracle_problem())
    if name == "c0":
        assert np.all(ref == 2e7)  # the literal aggregate terms cap every trial
    p = art.portfolio_from_workload(w, layouts=ALL_LAYOUTS)
    try:
        yet = device_yet(w)
        for v in VARIANTS:
            ylt, _ = run_ylt(p, w, v, yet=yet)
            y = ylt.cpu().numpy()
            assert_ylt_close(y, ref, gross, f"{name} variant {v}")
            mean, pml, tvar = gpu_metrics(ylt, [0.99])
            om, op, ot = oracle.metrics(ref, [0.99])
            np.testing.assert_allclose(pml, op, rtol=METRIC_RTOL)
            np.testing.assert_allclose(tvar, ot, rtol=METRIC_RTOL)
            np.testing.assert_allclose(mean, om, rtol=METRIC_RTOL)
    finally:
        p.close()


@pytest.fixture(scope="module")
def c1u():
    w = workloads.make("c1u")
    p = art.portfolio_from_workload(w)
    yet = device_yet(w)
    yield w, p, yet
    p.close()
    del yet
    torch.cuda.empty_cache()


def test_config1_sampled_plain_and_batched(c1u):
    """Paper scale (1e6 trials x 1000 events, 16 ELTs): the bench's launch,
    checked on 3000 sampled trials plus the first and last trial."""
    w, p, yet = c1u
    rng = np.random.default_rng(0)
    T = w.yet.n_trials
    trials = np.unique(np.concatenate([[0, T - 1], rng.choice(T, 3000, replace=False)]))
    ref, gross, _ = oracle_sample(w, trials)
    for v in (art.ART_VARIANT_PLAIN, art.ART_VARIANT_BATCHED, art.ART_VARIANT_SKIP, art.ART_VARIANT_SPARSE):
        ylt, _ = run_ylt(p, w, v, yet=yet)
        got = ylt[:, torch.from_numpy(trials).cuda()].cpu().numpy()
        assert_ylt_close(got, ref, gross, f"c1u variant {v}")
        assert torch.all(ylt >= 0) and torch.all(ylt <= w.portfolio.agg_lim[0])


def test_config1_full_ylt_against_oracle(c1u):
    """Every one of the 1,000,000 trials of the paper-scale one-layer
    workload (unsaturated terms): the skip variant the bench times and the
    plain one-layer-per-launch variant, element by element against the FP64
    oracle (about 1.6e10 lookups on the host cores)."""
    w, p, yet = c1u
    ref, gross, _ = oracle.ylt(w.oracle_problem())
    for v in (art.ART_VARIANT_SKIP, art.ART_VARIANT_PLAIN):
        ylt, _ = run_ylt(p, w, v, yet=yet)
        assert_ylt_close(ylt.cpu().numpy(), ref, gross, f"c1u variant {v}, all trials")


def test_config1_metrics_against_oracle_on_same_ylt(c1u):
    """The metrics kernels against the oracle's full-sort metrics on the same
    (GPU) YLT: the k-th largest is selected exactly."""
    w, p, yet = c1u
    ylt, _ = run_ylt(p, w, art.ART_VARIANT_BATCHED, yet=yet)
    probs = [0.99, 0.996, 0.999]
    mean, pml, tvar = gpu_metrics(ylt, probs)
    om, op, ot = oracle.metrics(ylt.cpu().numpy(), probs)
    np.testing.assert_array_equal(pml, op)
    np.testing.assert_allclose(tvar, ot, rtol=1e-12)
    np.testing.assert_allclose(mean, om, rtol=1e-12)


def test_literal_config1_caps_every_trial():
    w = workloads.make("c1", n_trials=20000)
    p = art.portfolio_from_workload(w)
    try:
        ylt, _ = run_ylt(p, w, art.ART_VARIANT_PLAIN)
        assert torch.all(ylt == 2e7)
        ref, gross, _ = oracle_sample(w, np.arange(0, 20000, 97))
        assert np.all(ref == 2e7)
    finally:
        p.close()


@pytest.mark.parametrize("variant,layouts", [
    ("ART_VARIANT_PLAIN", ALL_LAYOUTS), ("ART_VARIANT_BATCHED", ALL_LAYOUTS), ("ART_VARIANT_SKIP", ALL_LAYOUTS),
    ("ART_VARIANT_SPARSE", ALL_LAYOUTS), ("ART_VARIANT_FP64", ALL_LAYOUTS),
    ("ART_VARIANT_FP64", OCC64_LAYOUTS | art.ART_LAYOUT_SPARSE)])
def test_graph_replay_every_variant(variant, layouts):
    """ART_FLAG_GRAPH: the captured launches of each variant replay to the
    same bits as the direct call, and a new argument set re-captures."""
    w = workloads.random_case(204, catalogue=3001, n_elt=30, n_layers=21, n_trials=2500, max_len=80)
    v = getattr(art, variant)
    p = art.portfolio_from_workload(w, layouts=layouts)
    g = art.portfolio_from_workload(w, layouts=layouts, flags=art.ART_FLAG_GRAPH)
    try:
        ids, off, k, T = device_yet(w)
        L = w.portfolio.n_layers
        ref, _ = run_ylt(p, w, v)
        art.art_set_variant(g, v)
        for _ in range(3):
            y = torch.full((L, T), -1.0, dtype=torch.float64, device="cuda")
            art.art_run_ylt(g, T, ids, off, k, y)
            torch.cuda.synchronize()
            assert torch.equal(y, ref)
        # another YLT buffer and a shorter prefix: a new graph
        half = T // 2
        y2 = torch.full((L, half), -1.0, dtype=torch.float64, device="cuda")
        art.art_run_ylt(g, half, ids, None if off is None else off[:half + 1], k, y2)
        art.art_run_ylt(p, half, ids, None if off is None else off[:half + 1], k, y)
        torch.cuda.synchronize()
        # both calls wrote a [L][half] YLT; the direct one into the first L * half doubles of y
        assert torch.equal(y2.flatten(), y.flatten()[:L * half])
    finally:
        p.close()
        g.close()


def test_determinism_and_graph_replay():
    w = workloads.random_case(201, catalogue=2000, n_elt=20, n_layers=40, n_trials=3000, max_len=90)
    p = art.portfolio_from_workload(w)
    try:
        yet = device_yet(w)
        a, _ = run_ylt(p, w, art.ART_VARIANT_BATCHED, yet=yet)
        b, _ = run_ylt(p, w, art.ART_VARIANT_BATCHED, yet=yet)
        assert torch.equal(a, b)
        c, _ = run_ylt(p, w, art.ART_VARIANT_PLAIN, yet=yet)
        d, _ = run_ylt(p, w, art.ART_VARIANT_PLAIN, yet=yet)
        assert torch.equal(c, d)
        e, _ = run_ylt(p, w, art.ART_VARIANT_SKIP, yet=yet)
        f, _ = run_ylt(p, w, art.ART_VARIANT_SKIP, yet=yet)
        assert torch.equal(e, f)
        h, _ = run_ylt(p, w, art.ART_VARIANT_SPARSE, yet=yet)
        i, _ = run_ylt(p, w, art.ART_VARIANT_SPARSE, yet=yet)
        assert torch.equal(h, i)
    finally:
        p.close()
    g = art.portfolio_from_workload(w, flags=art.ART_FLAG_GRAPH)
    try:
        ids, off, k, T = device_yet(w)
        L = w.portfolio.n_layers
        outs = []
        for _ in range(3):
            y = torch.zeros((L, T), dtype=torch.float64, device="cuda") if not outs else outs[0]
            art.art_run_ylt(g, T, ids, off, k, y)
            torch.cuda.synchronize()
            outs.append(y.clone())
        assert torch.equal(outs[0], a) and torch.equal(outs[1], a) and torch.equal(outs[2], a)
    finally:
        g.close()


def test_host_buffers_match_device_path():
    """art_run_ylt_host (chunks of the YET copied from host memory, the YLT
    copied back) gives the device path's bits for every variant; the last
    workload spans two chunks."""
    cases = (workloads.random_case(202, n_trials=5000, max_len=80), workloads.make("c0u"),
             workloads.random_case(205, catalogue=20011, n_elt=12, n_layers=11, n_trials=50000, dense_k=400,
                                   nnz_frac=0.05))
    variants = [(art.ART_VARIANT_BATCHED, ALL_LAYOUTS), (art.ART_VARIANT_SKIP, ALL_LAYOUTS),
                (art.ART_VARIANT_SPARSE, ALL_LAYOUTS), (art.ART_VARIANT_PLAIN, ALL_LAYOUTS),
                (art.ART_VARIANT_FP64, OCC64_LAYOUTS | art.ART_LAYOUT_SPARSE)]
    for w in cases:
        for v, layouts in variants:
            p = art.portfolio_from_workload(w, layouts=layouts)
            try:
                dev, _ = run_ylt(p, w, v)
                L, T = w.portfolio.n_layers, w.yet.n_trials
                ids = torch.from_numpy(w.yet.event_ids).pin_memory()
                off = None if w.yet.trial_off is None else torch.from_numpy(w.yet.trial_off)
                out = torch.zeros((L, T), dtype=torch.float64).pin_memory()
                art.art_run_ylt_host(p, T, ids, off, w.yet.events_per_trial, out)
                assert torch.equal(out, dev.cpu()), (w.name, v)
            finally:
                p.close()


def _skip_ylt(w, layouts, layer_elt_ids=None):
    port = w.portfolio
    ids = port.layer_elt_ids if layer_elt_ids is None else layer_elt_ids
    tab = torch.from_numpy(port.elt_losses).cuda()
    terms = np.stack([port.occ_ret, port.occ_lim, port.agg_ret, port.agg_lim], axis=1)
    p = art.art_create_portfolio(port.catalogue_size, tab, port.elt_mult, port.elt_ded, port.elt_lim,
                                 port.layer_elt_off, ids, terms, layouts=layouts)
    try:
        y, _ = run_ylt(p, w, art.ART_VARIANT_SKIP)
        return y
    finally:
        p.close()


def test_occurrence_tables_from_csr_match_dense_build():
    """With the CSR of the non-zero losses the skip variant builds its
    occurrence tables from it; the YLT is that of the build from the
    per-layer tables, bit for bit, for layers listed in ascending ELT order,
    in descending order (events with three or more of a layer's entries
    re-summed from its per-layer row) and in c3's rotated order."""
    dense, csr = art.ART_LAYOUT_LAYER, art.ART_LAYOUT_LAYER | art.ART_LAYOUT_SPARSE
    cases = [(workloads.make("c0u"), None),
             (workloads.random_case(209, n_trials=4000, max_len=90, n_layers=11, n_elt=20, max_elts_per_layer=12,
                                    nnz_frac=0.6), None),
             (workloads.random_case(210, n_trials=3000, dense_k=200, n_layers=3, n_elt=9, nnz_frac=0.8), None),
             (workloads.make("c3", n_trials=3000), None)]
    w = cases[1][0]
    rev = w.portfolio.layer_elt_ids.copy()
    for j in range(w.portfolio.n_layers):
        a, b = w.portfolio.layer_elt_off[j], w.portfolio.layer_elt_off[j + 1]
        rev[a:b] = rev[a:b][::-1]
    cases.append((w, rev))
    w2 = cases[2][0]
    rev2 = w2.portfolio.layer_elt_ids.copy()
    for j in range(w2.portfolio.n_layers):
        a, b = w2.portfolio.layer_elt_off[j], w2.portfolio.layer_elt_off[j + 1]
        rev2[a:b] = np.roll(rev2[a:b], 1)
    cases.append((w2, rev2))
    for w, ids in cases:
        y_dense = _skip_ylt(w, dense, ids)
        y_csr = _skip_ylt(w, csr, ids)
        assert torch.equal(y_dense, y_csr), w.name
        prob = w.oracle_problem() if ids is None else dict(w.oracle_problem(), layer_elt_ids=ids)
        ref, gross, _ = oracle.ylt(prob)
        assert_ylt_close(y_csr.cpu().numpy(), ref, gross, f"{w.name} CSR build")


def test_host_buffers_in_place_and_staged():
    """The host-buffer calls read a mapped page-locked YET in place when the
    variant reads every id once (one occurrence group, or one layer for the
    plain variant), and stage it otherwise: pinned ids and offsets, the
    same with ART_FLAG_HOST_STAGED, and pageable buffers all give the device
    path's bits, with and without the metrics."""
    cases = (workloads.make("c0u"), workloads.random_case(208, n_trials=6000, max_len=90, n_layers=3))
    probs = [0.99]
    for w in cases:
        for v, layouts in ((art.ART_VARIANT_SKIP, art.ART_LAYOUT_LAYER),
                           (art.ART_VARIANT_FP64, OCC64_LAYOUTS | art.ART_LAYOUT_SPARSE),
                           (art.ART_VARIANT_PLAIN, art.ART_LAYOUT_LAYER)):
            p = art.portfolio_from_workload(w, layouts=layouts)
            try:
                dev, _ = run_ylt(p, w, v)
                mean, pml, tvar = gpu_metrics(dev, probs)
                L, T, K = w.portfolio.n_layers, w.yet.n_trials, w.yet.events_per_trial
                ids = torch.from_numpy(w.yet.event_ids)
                off = None if w.yet.trial_off is None else torch.from_numpy(w.yet.trial_off)
                for pinned, flags in ((True, 0), (True, art.ART_FLAG_HOST_STAGED), (False, 0)):
                    art.art_set_flags(p, flags)
                    i_h = ids.pin_memory() if pinned else ids.clone()
                    o_h = None if off is None else (off.pin_memory() if pinned else off.clone())
                    out = torch.zeros((L, T), dtype=torch.float64).pin_memory()
                    art.art_run_ylt_host(p, T, i_h, o_h, K, out)
                    assert torch.equal(out, dev.cpu()), (w.name, v, pinned, flags)
                    m, pm, tv = np.zeros(L), np.zeros((L, 1)), np.zeros((L, 1))
                    out.zero_()
                    art.art_run_ylt_host_metrics(p, T, i_h, o_h, K, probs, ylt=out, mean=m, pml=pm, tvar=tv)
                    assert torch.equal(out, dev.cpu()), (w.name, v, pinned, flags)
                    assert np.array_equal(m, mean) and np.array_equal(pm, pml) and np.array_equal(tv, tvar)
                assert art.art_get_device_status(p) == art.ART_OK
            finally:
                p.close()


def test_host_buffers_with_metrics_match_device_path():
    """art_run_ylt_host_metrics (YET from host memory, YLT kept on the device
    for the metrics) gives the bits of art_run_ylt followed by art_metrics,
    for a dense YET spanning two chunks and a ragged CSR one, with and
    without the YLT copied back."""
    cases = (workloads.random_case(206, catalogue=20011, n_elt=12, n_layers=11, n_trials=50000, dense_k=400,
                                   nnz_frac=0.05),
             workloads.random_case(207, n_trials=7000, max_len=90))
    probs = [0.9, 0.99, 0.999]
    for w in cases:
        p = art.portfolio_from_workload(w, layouts=ALL_LAYOUTS)
        try:
            dev, _ = run_ylt(p, w, art.ART_VARIANT_SKIP)
            mean, pml, tvar = gpu_metrics(dev, probs)
            L, T = w.portfolio.n_layers, w.yet.n_trials
            ids = torch.from_numpy(w.yet.event_ids).pin_memory()
            off = None if w.yet.trial_off is None else torch.from_numpy(w.yet.trial_off)
            for want_ylt in (True, False):
                out = torch.zeros((L, T), dtype=torch.float64).pin_memory() if want_ylt else None
                m = np.zeros(L)
                pm = np.zeros((L, len(probs)))
                tv = np.zeros((L, len(probs)))
                art.art_run_ylt_host_metrics(p, T, ids, off, w.yet.events_per_trial, probs, ylt=out, mean=m,
                                             pml=pm, tvar=tv)
                if want_ylt:
                    assert torch.equal(out, dev.cpu()), w.name
                assert np.array_equal(m, mean) and np.array_equal(pm, pml) and np.array_equal(tv, tvar), w.name
            om, op, ot = oracle.metrics(dev.cpu().numpy(), probs)
            np.testing.assert_array_equal(pm, op)
            np.testing.assert_allclose(tv, ot, rtol=1e-12)
        finally:
            p.close()


def test_l2_persist_flag_keeps_results():
    """ART_FLAG_L2_PERSIST (a persisting L2 window per occurrence group for
    the skip variant, over the pool table for the batched ones) changes no
    bit of the YLT, launched directly and from a captured graph."""
    w = workloads.random_case(208, catalogue=40009, n_elt=30, n_layers=19, n_trials=3000, max_len=200,
                              nnz_frac=0.05)
    ref_p = art.portfolio_from_workload(w, layouts=ALL_LAYOUTS)
    p = art.portfolio_from_workload(w, layouts=ALL_LAYOUTS, flags=art.ART_FLAG_L2_PERSIST)
    try:
        yet = device_yet(w)
        for v in (art.ART_VARIANT_SKIP, art.ART_VARIANT_BATCHED, art.ART_VARIANT_SPARSE):
            want, _ = run_ylt(ref_p, w, v, yet=yet)
            got, _ = run_ylt(p, w, v, yet=yet)
            assert torch.equal(got, want), v
            art.art_set_flags(p, art.ART_FLAG_L2_PERSIST | art.ART_FLAG_GRAPH)
            for _ in range(2):
                got, _ = run_ylt(p, w, v, yet=yet)
                assert torch.equal(got, want), ("graph", v)
            art.art_set_flags(p, art.ART_FLAG_L2_PERSIST)
    finally:
        p.close()
        ref_p.close()


def test_out_of_range_ids_flag_without_trapping():
    w = workloads.random_case(203, n_trials=50, min_len=5, max_len=20)
    ids = w.yet.event_ids.copy()
    ids[3] = w.portfolio.catalogue_size + 5
    ids[7] = -2
    bad = workloads.Workload(w.name, w.portfolio, workloads.YET(w.yet.n_trials, ids, 0, w.yet.trial_off), w.probs)
    p = art.portfolio_from_workload(w)
    try:
        for v in (art.ART_VARIANT_PLAIN, art.ART_VARIANT_BATCHED, art.ART_VARIANT_SKIP, art.ART_VARIANT_SPARSE):
            dids, off, k, T = device_yet(bad)
            art.art_set_variant(p, v)
            ylt = torch.zeros((w.portfolio.n_layers, T), dtype=torch.float64, device="cuda")
            art.art_run_ylt(p, T, dids, off, k, ylt)
            assert art.art_get_device_status(p) == art.ART_EID_RANGE
            assert art.art_get_device_status(p) == art.ART_OK  # the flag was cleared
            # bad events count as zero loss: same as the oracle with those ids on a zero row
            fixed = ids.copy()
            zero_ev = int(np.flatnonzero(w.portfolio.elt_losses.sum(axis=0) == 0)[0])
            fixed[3] = zero_ev
            fixed[7] = zero_ev
            ref, gross, _ = oracle.ylt(dict(w.oracle_problem(), event_ids=fixed))
            assert_ylt_close(ylt.cpu().numpy(), ref, gross, f"bad ids variant {v}")
    finally:
        p.close()


def test_decreasing_offsets_flag_einval():
    w = workloads.random_case(204, n_trials=20, min_len=3, max_len=9)
    off = w.yet.trial_off.copy()
    off[5], off[6] = off[6], off[5]
    p = art.portfolio_from_workload(w)
    try:
        ids = torch.from_numpy(w.yet.event_ids).cuda()
        doff = torch.from_numpy(off).cuda()
        ylt = torch.zeros((w.portfolio.n_layers, 20), dtype=torch.float64, device="cuda")
        art.art_run_ylt(p, 20, ids, doff, 0, ylt)
        assert art.art_get_device_status(p) == art.ART_EINVAL
    finally:
        p.close()


def test_update_terms_and_rounding():
    w = workloads.random_case(205, n_trials=300)
    p = art.portfolio_from_workload(w)
    try:
        m, d, l, t = art.art_get_terms(p)
        np.testing.assert_array_equal(m, w.portfolio.elt_mult)
        terms = t.copy()
        terms[:, 0] = terms[:, 0] * 1.7 + 0.1  # OccR: not FP32-representable in general
        art.art_update_terms(p, terms=terms)
        _, _, _, t2 = art.art_get_terms(p)
        np.testing.assert_array_equal(t2[:, 0], terms[:, 0].astype(np.float32).astype(np.float64))
        np.testing.assert_array_equal(t2[:, 2:], terms[:, 2:])
        prob = dict(w.oracle_problem(), occ_ret=t2[:, 0])
        ref, gross, _ = oracle.ylt(prob)
        for v in (art.ART_VARIANT_PLAIN, art.ART_VARIANT_BATCHED, art.ART_VARIANT_SKIP, art.ART_VARIANT_SPARSE):
            ylt, _ = run_ylt(p, w, v)
            assert_ylt_close(ylt.cpu().numpy(), ref, gross, f"updated terms variant {v}")
    finally:
        p.close()


def test_fp64_tables_rebuilt_and_repacked_keep_results():
    """Every all-FP64 call builds its occurrence tables and packs their entries
    in place. A catalogue past what shared memory holds folds the bitmap, and
    with every event carrying a loss each folded word is all ones, so the
    empty slots of partial chunks (mapped to the sentinel row C, which no
    build rewrites) gather row C: it must stay zero however often the tables
    are built and packed."""
    w = workloads.random_case(211, catalogue=2_000_003, n_elt=4, n_layers=4, n_trials=2000, min_len=1,
                              max_len=300, nnz_frac=1.0)
    w.portfolio.elt_ded[:] = 0.0  # every loss gives a positive payout
    w.portfolio.occ_ret[:] = 0.0  # every event with a loss has a positive occurrence loss
    ref, gross, _ = oracle.ylt(w.oracle_problem())
    p = art.portfolio_from_workload(w, layouts=OCC64_LAYOUTS)
    try:
        first, _ = run_ylt(p, w, art.ART_VARIANT_FP64)
        y = first.cpu().numpy()
        assert np.all(np.abs(y - ref) <= FP64_TOL * np.maximum(gross, 1.0))
        for _ in range(2):
            again, _ = run_ylt(p, w, art.ART_VARIANT_FP64)
            assert torch.equal(again, first)
        m, d, l, t = art.art_get_terms(p)
        art.art_update_terms(p, terms=np.column_stack([t[:, 0], t[:, 1] * 0.5, t[:, 2], t[:, 3]]))
        run_ylt(p, w, art.ART_VARIANT_FP64)
        art.art_update_terms(p, terms=t)
        back, _ = run_ylt(p, w, art.ART_VARIANT_FP64)
        assert torch.equal(back, first)
    finally:
        p.close()


@pytest.mark.parametrize("name,n_sample", [("c2", 5000), ("c4", 5000)])
def test_multilayer_workloads_sampled(name, n_sample):
    """The batching (CSR, 64 layers over a 256-ELT pool) and precision
    (128 layers over a 512-ELT pool) workloads at full size: every variant,
    checked on sampled trials, and the invariant 0 <= Y <= AggL on all."""
    w = workloads.make(name)
    p = art.portfolio_from_workload(w, layouts=ALL_LAYOUTS)
    try:
        yet = device_yet(w)
        T = w.yet.n_trials
        rng = np.random.default_rng(1)
        trials = np.unique(np.concatenate([[0, T - 1], rng.choice(T, n_sample, replace=False)]))
        ref, gross, _ = oracle_sample(w, trials)
        sel = torch.from_numpy(trials).cuda()
        for v in VARIANTS:
            ylt, _ = run_ylt(p, w, v, yet=yet)
            assert_ylt_close(ylt[:, sel].cpu().numpy(), ref, gross, f"{name} variant {v}")
            agg_lim = torch.from_numpy(w.portfolio.agg_lim).cuda()[:, None]
            assert torch.all(ylt >= 0) and torch.all(ylt <= agg_lim)
            del ylt
    finally:
        p.close()
    _check_fp64_occ(w, ref, gross, name, trials)


@pytest.mark.parametrize("name,n", [("c0", None), ("c0u", None), ("c1", 40000), ("c3", 8000)])
def test_early_exit_keeps_results(name, n):
    """The optional early exit of the skip and all-FP64 variants (stop
    reading a trial once it is capped) gives the oracle's results; on the
    literal one-layer terms, where every trial caps, exactly AggL."""
    w = workloads.make(name, n_trials=n)
    p = art.portfolio_from_workload(w)
    try:
        yet = device_yet(w)
        full, _ = run_ylt(p, w, art.ART_VARIANT_SKIP, yet=yet)
        art.art_set_flags(p, art.ART_FLAG_EARLY_EXIT)
        fast, _ = run_ylt(p, w, art.ART_VARIANT_SKIP, yet=yet)
        T = w.yet.n_trials
        trials = np.arange(0, T, max(1, T // 1500))
        ref, gross, _ = oracle_sample(w, trials)
        assert_ylt_close(fast[:, torch.from_numpy(trials).cuda()].cpu().numpy(), ref, gross, f"{name} early exit")
        capped = full == torch.from_numpy(w.portfolio.agg_lim).cuda()[:, None]
        assert torch.equal(fast[capped], full[capped])
        if name in ("c0", "c1"):
            assert torch.all(fast == 2e7)
        # the all-FP64 pass decides the cap on its exact fixed-point sums
        p64 = art.portfolio_from_workload(w, layouts=OCC64_LAYOUTS | art.ART_LAYOUT_SPARSE)
        try:
            art.art_set_flags(p64, art.ART_FLAG_EARLY_EXIT)
            y64, _ = run_ylt(p64, w, art.ART_VARIANT_FP64, yet=yet)
            y = y64[:, torch.from_numpy(trials).cuda()].cpu().numpy()
            assert np.all(np.abs(y - ref) <= FP64_TOL * np.maximum(gross, 1.0)), f"{name} all-FP64 early exit"
            if name in ("c0", "c1"):
                assert torch.all(y64 == 2e7)
        finally:
            p64.close()
    finally:
        p.close()

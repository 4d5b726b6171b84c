"""Degenerate and edge inputs through every forward variant and the metrics:
no events, no trials, no losses, one event, a catalogue that is not a
multiple of 32, repeated runs (determinism of the metrics)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1308_2572_gb300 import art, workloads

from gpu_util import assert_ylt_close, device_yet, gpu_metrics

pytestmark = pytest.mark.gpu

ALL = (art.ART_LAYOUT_LAYER | art.ART_LAYOUT_POOL | art.ART_LAYOUT_POOL64 | art.ART_LAYOUT_GROUP
       | art.ART_LAYOUT_SPARSE)
VARIANTS = [art.ART_VARIANT_PLAIN, art.ART_VARIANT_BATCHED, art.ART_VARIANT_FP64, art.ART_VARIANT_SKIP,
            art.ART_VARIANT_SPARSE]


def _run_all(w):
    ref, gross, _ = oracle.ylt(w.oracle_problem())
    p = art.portfolio_from_workload(w, layouts=ALL)
    try:
        ids, off, k, T = device_yet(w)
        L = w.portfolio.n_layers
        for v in VARIANTS:
            art.art_set_variant(p, v)
            y = torch.full((L, T), -5.0, dtype=torch.float64, device="cuda")
            art.art_run_ylt(p, T, ids, off, k, y)
            torch.cuda.synchronize()
            assert art.art_get_device_status(p) == art.ART_OK
            assert_ylt_close(y.cpu().numpy(), ref, gross, f"variant {v}")
    finally:
        p.close()
    # the all-FP64 variant over FP64 occurrence tables
    p = art.portfolio_from_workload(w, layouts=art.ART_LAYOUT_LAYER | art.ART_LAYOUT_OCC64)
    try:
        ids, off, k, T = device_yet(w)
        L = w.portfolio.n_layers
        art.art_set_variant(p, art.ART_VARIANT_FP64)
        y = torch.full((L, T), -5.0, dtype=torch.float64, device="cuda")
        art.art_run_ylt(p, T, ids, off, k, y)
        torch.cuda.synchronize()
        assert art.art_get_device_status(p) == art.ART_OK
        assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-12 * np.maximum(gross, 1.0))
    finally:
        p.close()
    return ref


def test_dense_trials_without_events():
    w = workloads.random_case(501, n_trials=100, dense_k=0)
    ref = _run_all(w)
    assert np.all(ref == 0)


def test_all_trials_empty_csr():
    """A CSR YET whose trials are all empty: the ABI wants a non-NULL id
    pointer for CSR input (it cannot read the offsets on the host), so one
    unused id stands behind it."""
    w = workloads.random_case(502, n_trials=64, min_len=0, max_len=0)
    assert w.yet.n_events == 0
    w = workloads.Workload(w.name, w.portfolio,
                           workloads.YET(w.yet.n_trials, np.zeros(1, np.int32), 0, w.yet.trial_off), w.probs)
    ref = _run_all(w)
    assert np.all(ref == 0)


def test_catalogue_not_a_multiple_of_32_and_ids_at_the_ends():
    w = workloads.random_case(503, catalogue=1037, n_trials=200, dense_k=40)
    ids = w.yet.event_ids.copy()
    ids[::7] = 1036       # last catalogue entry
    ids[3::11] = 0        # first
    w = workloads.Workload(w.name, w.portfolio, workloads.YET(w.yet.n_trials, ids, 40), w.probs)
    _run_all(w)


def test_no_losses_at_all_gives_zero():
    w = workloads.random_case(504, n_trials=50, dense_k=30)
    w.portfolio.elt_losses[:] = 0.0
    ref = _run_all(w)
    assert np.all(ref == 0)


def test_zero_trials_is_a_noop():
    w = workloads.random_case(505, n_trials=10, dense_k=5)
    p = art.portfolio_from_workload(w)
    try:
        ids, off, k, T = device_yet(w)
        y = torch.full((w.portfolio.n_layers, 1), 3.0, dtype=torch.float64, device="cuda")
        art.art_run_ylt(p, 0, ids, None, 5, y)
        torch.cuda.synchronize()
        assert torch.all(y == 3.0)
    finally:
        p.close()


def test_metrics_edges_and_determinism():
    g = torch.Generator(device="cpu").manual_seed(3)
    cases = [torch.zeros((2, 1), dtype=torch.float64),                         # one trial
             torch.full((3, 4097), 7.5, dtype=torch.float64),                  # all tied
             torch.rand((1, 123457), generator=g, dtype=torch.float64) * 1e9,  # ragged size
             torch.rand((3, 123458), generator=g, dtype=torch.float64) * 1e9,  # even length, ragged
             torch.tensor([[0.0, -0.0, 1.0, 5e-324, 1e300, 2.0]], dtype=torch.float64)]  # signed zero, subnormal
    for y in cases:
        yd = y.cuda().contiguous()
        probs = [0.5, 0.9, 0.99, 0.999999]
        a = gpu_metrics(yd, probs)
        b = gpu_metrics(yd, probs)
        for u, v in zip(a, b):
            assert np.array_equal(u, v)  # bitwise repeatable
        om, op, ot = oracle.metrics(np.abs(y.numpy()), probs)
        np.testing.assert_array_equal(a[1], op)
        np.testing.assert_allclose(a[2], ot, rtol=1e-12)
        np.testing.assert_allclose(a[0], om, rtol=1e-12)


@pytest.mark.parametrize("probs", [[0.5], [0.5, 0.9, 0.99, 0.999],
                                   [0.3, 0.45, 0.5, 0.55, 0.9, 0.99, 0.996, 0.999]])
def test_metrics_ties_decided_after_some_digits(probs):
    """Layers whose k-th largest loss sits in a block of equal losses among
    distinct losses sharing its leading bits: the candidates collapse to one
    key only after several radix digits, and the selection stops there. Next
    to a constant layer, a lognormal one and one capped above every quantile
    (with uncapped losses of the same binary exponent); PML exact, TVaR and
    mean within 1e-12 of the oracle's full sort, for 1, 4 and 8 probabilities."""
    rng = np.random.default_rng(11)
    n = 50021
    y = np.empty((5, n))
    y[0] = 2.0e7
    y[1] = rng.lognormal(10.0, 2.0, n)
    base = 1234.5
    y[2] = base * (1.0 + rng.uniform(-1e-9, 1e-9, n))      # same leading ~30 bits, distinct
    y[2, rng.choice(n, 6000, replace=False)] = base         # the ties straddle the median
    y[3] = np.where(rng.uniform(size=n) < 0.9995, 5.0e6, rng.uniform(4.2e6, 5.0e6, n))
    y[4] = np.where(rng.uniform(size=n) < 0.5, 0.0, 1.0)    # half zeros, half one value
    yd = torch.from_numpy(y).cuda().contiguous()
    a = gpu_metrics(yd, probs)
    b = gpu_metrics(yd, probs)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    om, op, ot = oracle.metrics(y, probs)
    np.testing.assert_array_equal(a[1], op)
    np.testing.assert_allclose(a[2], ot, rtol=1e-12)
    np.testing.assert_allclose(a[0], om, rtol=1e-12)
    assert np.all(a[1][2][np.asarray(probs) == 0.5] == base)


def test_metrics_with_and_without_candidate_lists_in_one_call():
    """Layers whose selected first-digit bucket holds every trial (uniform
    losses in [1, 1.25): one exponent, two leading mantissa bits; their
    candidate lists exceed the scratch and the layer reads its row in every
    pass) next to layers whose lists fit (lognormal, zero-heavy, capped with
    ties at the cap): PML exact, TVaR and mean within 1e-12 of the oracle's
    full sort, bitwise repeatable."""
    rng = np.random.default_rng(21)
    n = 300_007
    y = np.empty((6, n))
    y[0] = rng.uniform(1.0, 1.25, n)
    y[1] = rng.lognormal(12.0, 2.0, n)
    y[2] = rng.uniform(1.0, 1.25, n)
    y[3] = np.where(rng.uniform(size=n) < 0.7, 0.0, rng.lognormal(10.0, 1.0, n))
    y[4] = np.minimum(rng.lognormal(15.0, 1.5, n), 5.0e7)          # capped: ties at the largest key
    y[5] = np.where(rng.uniform(size=n) < 0.995, rng.uniform(0.0, 1e-310, n), 3.0)  # subnormals
    probs = [0.9, 0.99, 0.996, 0.999]
    yd = torch.from_numpy(y).cuda().contiguous()
    a = gpu_metrics(yd, probs)
    b = gpu_metrics(yd, probs)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    om, op, ot = oracle.metrics(y, probs)
    np.testing.assert_array_equal(a[1], op)
    np.testing.assert_allclose(a[2], ot, rtol=1e-12)
    np.testing.assert_allclose(a[0], om, rtol=1e-12)


def test_metrics_on_a_table_not_on_a_16_byte_boundary():
    """A table that starts 8 bytes past a 16-byte boundary (even row length):
    the metrics agree with the same table on an aligned copy and with the
    oracle."""
    torch.manual_seed(4)
    L, n = 3, 40002
    y = torch.distributions.LogNormal(10.0, 2.0).sample((L, n)).double()
    buf = torch.zeros(L * n + 2, dtype=torch.float64, device="cuda")
    off = buf[1:1 + L * n].view(L, n)
    off.copy_(y.cuda())
    assert off.data_ptr() % 16 == 8
    probs = [0.9, 0.99, 0.999]
    a = gpu_metrics(off, probs)
    b = gpu_metrics(y.cuda().contiguous(), probs)
    om, op, ot = oracle.metrics(y.numpy(), probs)
    for r in (a, b):
        np.testing.assert_array_equal(r[1], op)
        np.testing.assert_allclose(r[2], ot, rtol=1e-12)
        np.testing.assert_allclose(r[0], om, rtol=1e-12)


def test_catalogue_beyond_twice_the_shared_bitmap():
    """A catalogue of 4,000,037 events: the skip forward's and the group
    adjoint's bitmaps no longer fold into shared memory, so the upper events'
    bits are read from global memory. Dense (16-byte id loads) and CSR."""
    for dense_k, seed in ((64, 511), (None, 512)):
        w = workloads.random_case(seed, catalogue=4_000_037, n_elt=6, n_layers=5, n_trials=300, max_len=90,
                                  nnz_frac=0.05, dense_k=dense_k)
        ids = w.yet.event_ids
        assert ids.max() > 3_800_000 and ids.min() < 200_000
        _run_all(w)
        # the group adjoint against the per-layer adjoint on the same branch codes
        L, E, T = w.portfolio.n_layers, w.portfolio.n_elt, w.yet.n_trials
        pg = art.portfolio_from_workload(w, layouts=art.ART_LAYOUT_GROUP | art.ART_LAYOUT_LAYER)
        pl = art.portfolio_from_workload(w, layouts=art.ART_LAYOUT_LAYER)
        try:
            yet = device_yet(w)
            dids, off, k, _ = yet
            ylt = torch.empty((L, T), dtype=torch.float64, device="cuda")
            br = torch.empty((L, T), dtype=torch.uint8, device="cuda")
            art.art_set_variant(pl, art.ART_VARIANT_PLAIN)
            art.art_run_ylt(pl, T, dids, off, k, ylt, br)
            g = torch.full((L, T), 1.0 / T, dtype=torch.float64, device="cuda")
            outs = []
            for p in (pg, pl):
                gt = torch.empty((L, 4), dtype=torch.float64, device="cuda")
                gm = torch.empty(E, dtype=torch.float64, device="cuda")
                art.art_run_ylt_backward(p, T, dids, off, k, br, g, gt, gm)
                torch.cuda.synchronize()
                outs.append((gt.cpu().numpy(), gm.cpu().numpy()))
            np.testing.assert_allclose(outs[0][0], outs[1][0], rtol=1e-6, atol=1e-12)
            np.testing.assert_allclose(outs[0][1], outs[1][1], rtol=2e-6, atol=1e-9 * np.abs(outs[1][1]).max())
        finally:
            pg.close()
            pl.close()


def test_out_of_range_ids_dense_and_backward():
    """Ids outside [0, C) in a dense YET (16-byte id loads): every forward
    flags them and counts them as zero loss; both adjoints agree."""
    w = workloads.random_case(513, catalogue=1_037, n_trials=120, dense_k=40, n_layers=4)
    ids = w.yet.event_ids.copy()
    ids[[5, 77, 400, 4799]] = [w.portfolio.catalogue_size, -1, 2 ** 31 - 1, w.portfolio.catalogue_size + 3]
    bad = workloads.Workload(w.name, w.portfolio, workloads.YET(w.yet.n_trials, ids, 40, None), w.probs)
    zero_ev = int(np.flatnonzero(w.portfolio.elt_losses.sum(axis=0) == 0)[0])
    fixed = np.where((ids < 0) | (ids >= w.portfolio.catalogue_size), zero_ev, ids).astype(np.int32)
    ref, gross, _ = oracle.ylt(dict(w.oracle_problem(), event_ids=fixed))
    L, E, T = w.portfolio.n_layers, w.portfolio.n_elt, w.yet.n_trials
    p = art.portfolio_from_workload(w, layouts=ALL)
    pl = art.portfolio_from_workload(w, layouts=art.ART_LAYOUT_LAYER)
    try:
        dids, off, k, _ = device_yet(bad)
        for v in VARIANTS:
            art.art_set_variant(p, v)
            y = torch.zeros((L, T), dtype=torch.float64, device="cuda")
            art.art_run_ylt(p, T, dids, off, k, y)
            assert art.art_get_device_status(p) == art.ART_EID_RANGE, v
            assert_ylt_close(y.cpu().numpy(), ref, gross, f"bad dense ids, variant {v}")
        br = torch.empty((L, T), dtype=torch.uint8, device="cuda")
        y = torch.empty((L, T), dtype=torch.float64, device="cuda")
        art.art_set_variant(pl, art.ART_VARIANT_PLAIN)
        art.art_run_ylt(pl, T, dids, off, k, y, br)
        art.art_get_device_status(pl)
        g = torch.full((L, T), 1.0 / T, dtype=torch.float64, device="cuda")
        outs = []
        for q in (p, pl):
            gt = torch.empty((L, 4), dtype=torch.float64, device="cuda")
            gm = torch.empty(E, dtype=torch.float64, device="cuda")
            art.art_run_ylt_backward(q, T, dids, off, k, br, g, gt, gm)
            torch.cuda.synchronize()
            outs.append((gt.cpu().numpy(), gm.cpu().numpy()))
        np.testing.assert_allclose(outs[0][0], outs[1][0], rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(outs[0][1], outs[1][1], rtol=2e-6, atol=1e-12)
        ot, om, _, _ = oracle.grad(dict(w.oracle_problem(), event_ids=fixed), g.cpu().numpy())
        np.testing.assert_allclose(outs[0][0], ot, rtol=1e-6, atol=1e-9)
    finally:
        p.close()
        pl.close()

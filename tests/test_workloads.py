"""The seeded synthetic inputs against their stated recipe (CPU).

Every parity case and bench line runs on these generators, which stand in
for the paper's proprietary YET and ELTs (Sections II and III: a catalogue
of 2,000,000 events, 1,000,000 trials of about 1,000 events, ELTs as
direct-access tables of 10,000-50,000 non-zero losses). The checks pin the
shapes, value ranges, distributions, terms and seeding; the two pools of
hundreds of ELTs (2-4 GB of tables) are left to the GPU tests.
"""
import numpy as np
import pytest

from paper_1308_2572_gb300 import workloads


@pytest.fixture(scope="module")
def c0():
    return workloads.make("c0")


def test_c0_shapes_and_ids(c0):
    p, y = c0.portfolio, c0.yet
    assert p.catalogue_size == 100_000
    assert y.n_trials == 10_000 and y.events_per_trial == 1000 and y.trial_off is None
    assert y.event_ids.dtype == np.int32 and y.event_ids.size == 10_000 * 1000
    assert y.event_ids.min() >= 0 and y.event_ids.max() < 100_000
    # uniform with replacement: every id bin about equally full
    counts = np.bincount(y.event_ids, minlength=100_000)
    assert abs(counts.mean() - 100.0) < 1e-9 and counts.std() < 12.0


def test_c0_tables_and_terms(c0):
    p = c0.portfolio
    assert p.elt_losses.shape == (3, 100_000) and p.elt_losses.dtype == np.float32
    for e in range(3):
        nz = p.elt_losses[e][p.elt_losses[e] > 0]
        assert nz.size == 10_000
        logs = np.log(nz.astype(np.float64))
        assert abs(logs.mean() - 12.0) < 0.1 and abs(logs.std() - 2.0) < 0.1
        # deductible and limit: 5th and 99th percentiles of the non-zero losses
        assert p.elt_ded[e] == np.float32(np.percentile(nz.astype(np.float64), 5))
        assert p.elt_lim[e] == np.float32(np.percentile(nz.astype(np.float64), 99))
    assert np.all(p.elt_mult == 1.0)
    assert list(p.layer_elt_off) == [0, 3] and list(p.layer_elt_ids) == [0, 1, 2]
    assert (p.occ_ret[0], p.occ_lim[0], p.agg_ret[0], p.agg_lim[0]) == (1e5, 5e6, 1e6, 2e7)
    assert list(c0.probs) == [0.99]


def test_unsaturated_variants_change_only_the_aggregate_terms(c0):
    u = workloads.make("c0u")
    assert np.array_equal(u.yet.event_ids, c0.yet.event_ids)
    assert np.array_equal(u.portfolio.elt_losses, c0.portfolio.elt_losses)
    assert (u.portfolio.agg_ret[0], u.portfolio.agg_lim[0]) == (1.5e8, 1e8)


def test_seeding_is_reproducible_and_prefixes_agree():
    a = workloads.make("c1", n_trials=20)
    b = workloads.make("c1", n_trials=20)
    c = workloads.make("c1", n_trials=50)
    assert np.array_equal(a.yet.event_ids, b.yet.event_ids)
    assert np.array_equal(a.portfolio.elt_losses, b.portfolio.elt_losses)
    # a smaller trial count keeps the first trials of the full YET
    assert np.array_equal(a.yet.event_ids, c.yet.event_ids[:20 * 1000])
    p = a.portfolio
    assert p.catalogue_size == 2_000_000 and p.elt_losses.shape == (16, 2_000_000)
    assert all(int((p.elt_losses[e] > 0).sum()) == 20_000 for e in range(16))
    assert a.yet.event_ids.max() < 2_000_000


def test_c3_layer_structure():
    w = workloads.make("c3", n_trials=10)
    p = w.portfolio
    assert p.n_layers == 8
    for j in range(8):
        elts = list(p.layer_elt_ids[p.layer_elt_off[j]:p.layer_elt_off[j + 1]])
        assert elts == [(2 * j + i) % 16 for i in range(8)]
        assert p.agg_ret[j] == 3e7 + 5e6 * j and p.agg_lim[j] == 3e7
        assert p.occ_ret[j] == 1e5 and p.occ_lim[j] == 5e6
    assert np.all(p.elt_mult == 1.0)


def test_random_cases_are_seeded():
    a = workloads.random_case(5)
    b = workloads.random_case(5)
    c = workloads.random_case(6)
    assert np.array_equal(a.yet.event_ids, b.yet.event_ids)
    assert not np.array_equal(a.portfolio.elt_losses, c.portfolio.elt_losses)


def _branches(name, n_trials=None):
    import oracle  # test infrastructure: the FP64 reference
    w = workloads.make(name, n_trials=n_trials)
    y = oracle.ylt(w.oracle_problem())[0]
    lim = w.portfolio.agg_lim[:, None]
    zero, cap = (y == 0).mean(axis=1), (y == lim).mean(axis=1)
    return zero, 1.0 - zero - cap, cap, ((y > 0) & (y < lim)).any(axis=0).mean()


def test_parity_workloads_reach_every_aggregate_branch():
    """The unsaturated and multi-layer workloads put trials on all three
    pieces of the aggregate terms (zero, middle, capped), so parity and
    gradient tests exercise each; the literal one-layer terms cap every
    trial."""
    zero, mid, cap, any_mid = _branches("c3", 2000)
    assert any_mid > 0.9                      # nearly every trial is on some layer's middle piece
    assert np.all(mid > 0.05)
    assert cap[0] > 0.05 and zero[-1] > 0.5   # low layers cap often, high layers rarely attach
    zero, mid, cap, _ = _branches("c1u", 2000)
    assert zero[0] > 0.1 and mid[0] > 0.5 and cap[0] > 0.005
    zero, mid, cap, _ = _branches("c1", 500)
    assert cap[0] == 1.0


@pytest.mark.parametrize("name", ["c2", "c4"])
def test_pool_workloads_spread_over_the_aggregate_branches(name):
    """The log-uniform layer terms of the pool workloads leave about a
    quarter of (layer, trial) results at zero, a quarter capped and half in
    between, with most layers at least 10% in between."""
    zero, mid, cap, _ = _branches(name, 300)
    assert 0.15 < zero.mean() < 0.4 and 0.15 < cap.mean() < 0.4 and mid.mean() > 0.35
    assert (mid >= 0.1).mean() > 0.45


def test_shards_share_the_portfolio_and_draw_their_own_yet():
    """shard 0 is the workload itself; shard s > 0 keeps the portfolio and
    draws another YET of the same recipe, reproducibly."""
    a = workloads.make("c0u", n_trials=300)
    b = workloads.make("c0u", n_trials=300, shard=0)
    c = workloads.make("c0u", n_trials=300, shard=1)
    c2 = workloads.make("c0u", n_trials=300, shard=1)
    d = workloads.make("c0u", n_trials=300, shard=2)
    assert np.array_equal(a.yet.event_ids, b.yet.event_ids)
    assert np.array_equal(c.yet.event_ids, c2.yet.event_ids)
    assert not np.array_equal(a.yet.event_ids, c.yet.event_ids)
    assert not np.array_equal(c.yet.event_ids, d.yet.event_ids)
    for w in (c, d):
        assert np.array_equal(w.portfolio.elt_losses, a.portfolio.elt_losses)
        assert np.array_equal(w.portfolio.agg_ret, a.portfolio.agg_ret)
        assert w.yet.event_ids.shape == a.yet.event_ids.shape
        assert w.yet.event_ids.min() >= 0 and w.yet.event_ids.max() < a.portfolio.catalogue_size

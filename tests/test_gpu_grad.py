"""GPU parity for the adjoint (art_metrics_backward + art_run_ylt_backward)
and the torch.autograd.Function around it.

Workload: the 8-layer, 16-ELT portfolio over the paper-scale YET, first
10,000 trials. The objective is sum_j (EL_j + TVaR_0.99,j). Checked against
the FP64 oracle's analytic gradient (weights built here from the oracle's
own YLT) and against central differences of the GPU forward.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1308_2572_gb300 import art, workloads
from paper_1308_2572_gb300.autograd import layer_metrics

from gpu_util import device_yet

pytestmark = pytest.mark.gpu

N_TRIALS = 10_000
PROB = 0.99


# the adjoint reads the group tables when they exist (one pass per layer
# group), else the per-layer tables (one pass per layer): both are checked
LAYOUTS = {"group": art.ART_LAYOUT_LAYER | art.ART_LAYOUT_GROUP, "layer": art.ART_LAYOUT_LAYER}


@pytest.fixture(scope="module", params=sorted(LAYOUTS))
def c3(request):
    w = workloads.make("c3", n_trials=N_TRIALS)
    p = art.portfolio_from_workload(w, layouts=LAYOUTS[request.param])
    yet = device_yet(w)
    yield w, p, yet
    p.close()


def _oracle_weights(y_ref, k):
    """dObjective/dY for sum_j (mean_j + TVaR_j) from the oracle's YLT: 1/N,
    plus 1/k above the k-th largest, ties at it sharing the remainder."""
    L, N = y_ref.shape
    g = np.full((L, N), 1.0 / N)
    for j in range(L):
        s = np.sort(y_ref[j])[::-1]
        pml = s[k - 1]
        gt = y_ref[j] > pml
        eq = y_ref[j] == pml
        g[j, gt] += 1.0 / k
        g[j, eq] += (k - gt.sum()) / (k * eq.sum())
    return g


def _gpu_grad(p, yet, L, n_elt):
    ids, off, K, T = yet
    ylt = torch.empty((L, T), dtype=torch.float64, device="cuda")
    br = torch.empty((L, T), dtype=torch.uint8, device="cuda")
    art.art_set_variant(p, art.ART_VARIANT_PLAIN)
    art.art_run_ylt(p, T, ids, off, K, ylt, br)
    mean = torch.empty(L, dtype=torch.float64, device="cuda")
    pml = torch.empty((L, 1), dtype=torch.float64, device="cuda")
    tvar = torch.empty((L, 1), dtype=torch.float64, device="cuda")
    art.art_metrics(ylt, T, L, [PROB], mean, pml, tvar)
    gy = torch.empty_like(ylt)
    ones = torch.ones(L, dtype=torch.float64, device="cuda")
    art.art_metrics_backward(ylt, T, L, [PROB], pml, ones, ones.reshape(L, 1).contiguous(), gy)
    gt = torch.empty((L, 4), dtype=torch.float64, device="cuda")
    gm = torch.empty(n_elt, dtype=torch.float64, device="cuda")
    art.art_run_ylt_backward(p, T, ids, off, K, br, gy, gt, gm)
    torch.cuda.synchronize()
    return ylt.cpu().numpy(), br.cpu().numpy(), gy.cpu().numpy(), gt.cpu().numpy(), gm.cpu().numpy(), mean, tvar


def test_branch_codes_match_oracle_aggregate(c3):
    w, p, yet = c3
    L = w.portfolio.n_layers
    ylt, br, *_ = _gpu_grad(p, yet, L, w.portfolio.n_elt)
    _, _, s = oracle.ylt(w.oracle_problem(), want_sum=True)
    ar, al = w.portfolio.agg_ret[:, None], w.portfolio.agg_lim[:, None]
    expect = np.where(s <= ar, 0, np.where(s - ar > al, 2, 1))
    mism = br != expect
    # a mismatch is only allowed where the FP64 aggregate sits within FP32
    # rounding of a kink
    near = (np.abs(s - ar) <= 1e-6 * s) | (np.abs(s - ar - al) <= 1e-6 * s)
    assert not np.any(mism & ~near)
    assert 0.05 < np.mean(expect == 1) < 0.95  # the portfolio exercises every branch
    assert np.any(expect == 2) and np.any(expect == 0)


def test_gradient_matches_oracle(c3):
    w, p, yet = c3
    L, E = w.portfolio.n_layers, w.portfolio.n_elt
    k = oracle.tail_count(PROB, N_TRIALS)
    _, _, _, gt, gm, _, _ = _gpu_grad(p, yet, L, E)
    y_ref, gross, _ = oracle.ylt(w.oracle_problem())
    g = _oracle_weights(y_ref, k)
    ot, om, _, _ = oracle.grad(w.oracle_problem(), g)
    np.testing.assert_allclose(gt, ot, rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(gm, om, rtol=1e-6, atol=1e-3)
    assert np.all(gt[:, 2] <= 0) and np.all(gt[:, 0] <= 0)  # retentions lower the losses
    assert np.all(gm >= 0)


def test_gradient_matches_gpu_central_differences(c3):
    """dObjective/dtheta against (Obj(theta + h) - Obj(theta - h)) / 2h of the
    GPU forward, h = 1e-4 |theta| (the FP32-rounded step for FP32 terms)."""
    w, p, yet = c3
    L, E = w.portfolio.n_layers, w.portfolio.n_elt
    _, _, _, gt, gm, _, _ = _gpu_grad(p, yet, L, E)
    m0, d0, l0, t0 = art.art_get_terms(p)
    ids, off, K, T = yet

    def objective():
        ylt = torch.empty((L, T), dtype=torch.float64, device="cuda")
        art.art_run_ylt(p, T, ids, off, K, ylt)
        mean = torch.empty(L, dtype=torch.float64, device="cuda")
        pml = torch.empty((L, 1), dtype=torch.float64, device="cuda")
        tvar = torch.empty((L, 1), dtype=torch.float64, device="cuda")
        art.art_metrics(ylt, T, L, [PROB], mean, pml, tvar)
        return float(mean.sum() + tvar.sum())

    checked = 0
    try:
        for j in range(0, L, 3):
            for c in range(4):
                tp, tm = t0.copy(), t0.copy()
                h = 1e-4 * abs(t0[j, c])
                tp[j, c] += h
                tm[j, c] -= h
                art.art_update_terms(p, terms=tp)
                _, _, _, tpr = art.art_get_terms(p)
                fp = objective()
                art.art_update_terms(p, terms=tm)
                _, _, _, tmr = art.art_get_terms(p)
                fm = objective()
                fd = (fp - fm) / (tpr[j, c] - tmr[j, c])
                assert fd == pytest.approx(gt[j, c], rel=2e-3, abs=1e-3 * max(1.0, abs(gt[j, c]))), (j, c)
                checked += 1
            art.art_update_terms(p, terms=t0)
        for e in range(0, E, 5):
            mp, mm = m0.copy(), m0.copy()
            mp[e] *= 1 + 1e-4
            mm[e] *= 1 - 1e-4
            art.art_update_terms(p, elt_mult=mp)
            mpr = art.art_get_terms(p)[0]
            fp = objective()
            art.art_update_terms(p, elt_mult=mm)
            mmr = art.art_get_terms(p)[0]
            fm = objective()
            fd = (fp - fm) / (float(mpr[e]) - float(mmr[e]))
            assert fd == pytest.approx(gm[e], rel=2e-3), e
            checked += 1
    finally:
        art.art_update_terms(p, elt_mult=m0, terms=t0)
    assert checked >= 12


def test_autograd_function(c3):
    w, p, yet = c3
    L, E = w.portfolio.n_layers, w.portfolio.n_elt
    art.art_set_variant(p, art.ART_VARIANT_PLAIN)
    m0, _, _, t0 = art.art_get_terms(p)
    params = [torch.tensor(t0[:, c], dtype=torch.float64, requires_grad=True) for c in range(4)]
    mult = torch.tensor(m0.astype(np.float64), requires_grad=True)
    mean, tvar = layer_metrics(p, yet, [PROB], *params, mult)
    (mean.sum() + tvar.sum()).backward()
    _, _, _, gt, gm, gmean, gtvar = _gpu_grad(p, yet, L, E)
    np.testing.assert_allclose(mean.detach().numpy(), gmean.cpu().numpy(), rtol=0, atol=0)
    for c in range(4):
        np.testing.assert_allclose(params[c].grad.numpy(), gt[:, c], rtol=1e-12, atol=0)
    np.testing.assert_allclose(mult.grad.numpy(), gm, rtol=1e-12, atol=0)


def test_autograd_backward_uses_its_own_forward_terms(c3):
    """forward(A), forward(B), backward of A: the gradient is A's (against the
    oracle's analytic gradient at A's terms), and the portfolio keeps B's terms."""
    w, p, yet = c3
    L, E = w.portfolio.n_layers, w.portfolio.n_elt
    art.art_set_variant(p, art.ART_VARIANT_PLAIN)
    m0, _, _, t0 = art.art_get_terms(p)
    try:
        pa = [torch.tensor(t0[:, c], dtype=torch.float64, requires_grad=True) for c in range(4)]
        ma = torch.tensor(m0.astype(np.float64), requires_grad=True)
        mean_a, tvar_a = layer_metrics(p, yet, [PROB], *pa, ma)
        # scenario B: other retentions and multipliers, forward only
        tb = t0.copy()
        tb[:, 0] *= 1.5
        tb[:, 2] *= 0.8
        mb = (m0 * np.float32(1.1)).astype(np.float64)
        pb = [torch.tensor(tb[:, c], dtype=torch.float64, requires_grad=True) for c in range(4)]
        layer_metrics(p, yet, [PROB], *pb, torch.tensor(mb, requires_grad=True))
        after_b = art.art_get_terms(p)
        (mean_a.sum() + tvar_a.sum()).backward()
        # the portfolio is left with B's terms
        assert all(np.array_equal(x, y) for x, y in zip(art.art_get_terms(p), after_b))
        k = oracle.tail_count(PROB, N_TRIALS)
        y_ref, _, _ = oracle.ylt(w.oracle_problem())
        ot, om, _, _ = oracle.grad(w.oracle_problem(), _oracle_weights(y_ref, k))
        got = np.stack([pa[c].grad.numpy() for c in range(4)], axis=1)
        np.testing.assert_allclose(got, ot, rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(ma.grad.numpy(), om, rtol=1e-6, atol=1e-3)
    finally:
        art.art_update_terms(p, elt_mult=m0, terms=t0)


def _adjoint(p, yet, br, g, L, n_elt):
    ids, off, K, T = yet
    gt = torch.empty((L, 4), dtype=torch.float64, device="cuda")
    gm = torch.empty(n_elt, dtype=torch.float64, device="cuda")
    art.art_run_ylt_backward(p, T, ids, off, K, br, g, gt, gm)
    torch.cuda.synchronize()
    return gt.cpu().numpy(), gm.cpu().numpy()


def test_group_adjoint_many_groups_matches_layer_adjoint_and_oracle():
    """Several layer groups sharing ELTs (a multiplier's gradient sums over
    groups), ragged trials, random weights: the group adjoint against the
    per-layer adjoint (same branch codes) and against the oracle."""
    w = workloads.random_case(601, catalogue=3001, n_elt=40, n_layers=30, n_trials=4000, max_len=100,
                              max_elts_per_layer=12, mult_range=(0.8, 1.25))
    L, E, T = w.portfolio.n_layers, w.portfolio.n_elt, w.yet.n_trials
    pg = art.portfolio_from_workload(w, layouts=art.ART_LAYOUT_GROUP | art.ART_LAYOUT_LAYER)
    pl = art.portfolio_from_workload(w, layouts=art.ART_LAYOUT_LAYER)
    try:
        yet = device_yet(w)
        ids, off, K, _ = yet
        rng = np.random.Generator(np.random.PCG64(602))
        g_host = rng.uniform(0.0, 2.0, size=(L, T)) / T
        g_host[:, ::7] = 0.0  # trials without weight are skipped
        g = torch.from_numpy(g_host).cuda()
        ylt = torch.empty((L, T), dtype=torch.float64, device="cuda")
        br = torch.empty((L, T), dtype=torch.uint8, device="cuda")
        art.art_set_variant(pl, art.ART_VARIANT_PLAIN)
        art.art_run_ylt(pl, T, ids, off, K, ylt, br)
        assert len({int(x) for x in np.unique(br.cpu().numpy())}) == 3
        gt_g, gm_g = _adjoint(pg, yet, br, g, L, E)
        gt_l, gm_l = _adjoint(pl, yet, br, g, L, E)
        # the group path rounds each weight g to FP32 once (relative 2^-24 per
        # term); the per-layer path applies it in FP64
        np.testing.assert_allclose(gt_g, gt_l, rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(gm_g, gm_l, rtol=2e-6, atol=1e-9 * np.abs(gm_l).max())
        ot, om, _, _ = oracle.grad(w.oracle_problem(), g_host)
        np.testing.assert_allclose(gt_g, ot, rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(gm_g, om, rtol=2e-6, atol=1e-9 * np.abs(om).max())
        # deterministic: a second run gives the same bits
        gt2, gm2 = _adjoint(pg, yet, br, g, L, E)
        assert np.array_equal(gt2, gt_g) and np.array_equal(gm2, gm_g)
    finally:
        pg.close()
        pl.close()


def test_backward_needs_group_or_layer_tables():
    w = workloads.random_case(603, n_trials=20)
    p = art.portfolio_from_workload(w, layouts=art.ART_LAYOUT_POOL)
    try:
        ids, off, K, T = device_yet(w)
        L, E = w.portfolio.n_layers, w.portfolio.n_elt
        br = torch.zeros((L, T), dtype=torch.uint8, device="cuda")
        g = torch.zeros((L, T), dtype=torch.float64, device="cuda")
        gt = torch.empty((L, 4), dtype=torch.float64, device="cuda")
        gm = torch.empty(E, dtype=torch.float64, device="cuda")
        with pytest.raises(art.ArtError) as ei:
            art.art_run_ylt_backward(p, T, ids, off, K, br, g, gt, gm)
        assert ei.value.status == art.ART_EUNSUPPORTED
    finally:
        p.close()

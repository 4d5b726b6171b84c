"""Trial-sharded metrics on one GPU: the YET split into ranges, each range's
forward and art_topk run in turn (as each GPU of a sharded run would run its
own), the lists merged on the host (art_merge_topk). Against art_metrics on
the unsplit YLT (PML bit for bit, TVaR and mean within 1e-12) and the
oracle; art_topk's lists against the layout it documents."""
import numpy as np
import pytest
import torch

import oracle
from paper_1308_2572_gb300 import art, shard, workloads

from gpu_util import assert_ylt_close, device_yet, gpu_metrics, run_ylt

pytestmark = pytest.mark.gpu


def _shard_yet(w, ids, t0, t1):
    """Device YET of trials [t0, t1): a view of the ids, rebased offsets."""
    if w.yet.trial_off is None:
        K = w.yet.events_per_trial
        return ids[t0 * K:t1 * K], None, K, t1 - t0
    off = w.yet.trial_off
    o = torch.from_numpy(off[t0:t1 + 1] - off[t0]).cuda()
    return ids[int(off[t0]):int(off[t1])], o, 0, t1 - t0


@pytest.mark.parametrize("name,n_shards,probs", [("c0u", 3, [0.99]), ("ragged", 4, [0.9, 0.99, 0.999]),
                                                 ("c2", 2, [0.99, 0.996])])
def test_sharded_metrics_match_the_unsplit_ylt(name, n_shards, probs):
    if name == "ragged":
        w = workloads.random_case(1501, catalogue=3001, n_elt=20, n_layers=9, n_trials=20011, max_len=120)
    elif name == "c2":
        w = workloads.make("c2", n_trials=30000)
    else:
        w = workloads.make(name)
    p = art.portfolio_from_workload(w)
    try:
        ids, off, K, T = device_yet(w)
        L = w.portfolio.n_layers
        full, _ = run_ylt(p, w, art.ART_VARIANT_SKIP, yet=(ids, off, K, T))
        mean, pml, tvar = gpu_metrics(full, probs)
        k = shard.list_length(T, probs)
        tops, sums, parts = [], [], []
        for r in range(n_shards):
            t0, t1 = shard.trial_range(T, n_shards, r)
            y = torch.empty((L, t1 - t0), dtype=torch.float64, device="cuda")
            art.art_run_ylt(p, t1 - t0, *_shard_yet(w, ids, t0, t1)[:3], y)
            top = torch.empty((L, k), dtype=torch.float64, device="cuda")
            sm = torch.empty(L, dtype=torch.float64, device="cuda")
            art.art_topk(y, t1 - t0, L, k, top, sm)
            torch.cuda.synchronize()
            tops.append(top.cpu().numpy())
            sums.append(sm.cpu().numpy())
            parts.append(y.cpu().numpy())
        assert art.art_get_device_status(p) == art.ART_OK
        # the shards' rows are the unsplit YLT's columns
        assert np.array_equal(np.concatenate(parts, axis=1), full.cpu().numpy())
        m2, p2, t2 = shard.merge(np.stack(tops), np.stack(sums), T, probs)
        np.testing.assert_array_equal(p2, pml)
        np.testing.assert_allclose(t2, tvar, rtol=1e-12)
        np.testing.assert_allclose(m2, mean, rtol=1e-12)
        om, op, ot = oracle.metrics(full.cpu().numpy(), probs)
        np.testing.assert_array_equal(p2, op)
        np.testing.assert_allclose(t2, ot, rtol=1e-12)
    finally:
        p.close()


def test_topk_lists_follow_their_documented_layout():
    rng = np.random.default_rng(15)
    n = 70001
    y = np.stack([rng.lognormal(11.0, 2.0, n), np.where(rng.uniform(size=n) < 0.5, 0.0, 7.0),
                  np.full(n, 3.0), rng.uniform(0.0, 1.0, n)])
    yd = torch.from_numpy(y).cuda().contiguous()
    L = y.shape[0]
    for k in (1, 700, 50000, 100000):  # the last longer than the table
        top = torch.full((L, k), -1.0, dtype=torch.float64, device="cuda")
        sm = torch.empty(L, dtype=torch.float64, device="cuda")
        art.art_topk(yd, n, L, k, top, sm)
        a = top.cpu().numpy()
        art.art_topk(yd, n, L, k, top, sm)
        assert np.array_equal(a, top.cpu().numpy())  # deterministic
        ke = min(k, n)
        for j in range(L):
            thr = np.sort(y[j])[::-1][ke - 1]
            above = y[j][y[j] > thr]
            want = np.zeros(k)
            want[:above.size] = above          # in trial order
            want[above.size:ke] = thr
            assert np.array_equal(a[j], want), (k, j)
        np.testing.assert_allclose(sm.cpu().numpy(), y.sum(axis=1), rtol=1e-12)

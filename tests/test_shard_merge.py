"""Trial-sharded metrics on CPU: two gloo ranks each reduce their share of
an oracle YLT to top-k lists and sums, the lists are all-gathered, and the
library's host merge (art_merge_topk, no GPU needed) gives the whole YLT's
PML bit for bit and its TVaR and mean within 1e-12 of the oracle's full
sort. The per-shard lists are made here with numpy in the layout art_topk
documents (its GPU kernel is checked against the same layout in
tests/test_gpu_shard.py)."""
import os
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1308_2572_gb300 import shard, workloads  # noqa: E402

PROBS = [0.9, 0.99, 0.996, 0.999]


def shard_list(y, k):
    """art_topk's documented list for rows y [L][T]: the losses above the
    min(k, T)-th largest in trial order, that loss repeated up to min(k, T)
    entries, then zeros up to k; and the rows' sums."""
    L, T = y.shape
    ke = min(k, T)
    top = np.zeros((L, k))
    for j in range(L):
        thr = np.sort(y[j])[::-1][ke - 1]
        above = y[j][y[j] > thr]
        top[j, :above.size] = above
        top[j, above.size:ke] = thr
    return top, y.sum(axis=1)


def _ylt():
    w = workloads.random_case(1401, catalogue=499, n_elt=9, n_layers=6, n_trials=3001, max_len=60)
    y, _, _ = oracle.ylt(w.oracle_problem(), want_gross=False)
    return y


def _worker(rank, world, port, y, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        T = y.shape[1]
        t0, t1 = shard.trial_range(T, world, rank)
        k = shard.list_length(T, PROBS)
        top, sums = shard_list(y[:, t0:t1], k)
        top_all, sums_all = shard.gather_lists(torch.from_numpy(top), torch.from_numpy(sums))
        out[rank] = shard.merge(top_all, sums_all, T, PROBS)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_merge_to_the_whole_ylt_metrics():
    y = _ylt()
    port = 29600 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, y, out), nprocs=2, join=True)
        res = dict(out)
    om, op, ot = oracle.metrics(y, PROBS)
    for rank in (0, 1):
        mean, pml, tvar = res[rank]
        np.testing.assert_array_equal(pml, op)
        np.testing.assert_allclose(tvar, ot, rtol=1e-12)
        np.testing.assert_allclose(mean, om, rtol=1e-12)
    assert all(np.array_equal(a, b) for a, b in zip(res[0], res[1]))  # every rank the same bits


@pytest.mark.parametrize("n_shards", [1, 3, 7])
def test_merge_of_uneven_shards_including_shards_shorter_than_k(n_shards):
    y = _ylt()
    T = y.shape[1]
    probs = [0.5, 0.99]  # k = 1501 at p = 0.5: longer than a 7-way shard
    k = shard.list_length(T, probs)
    tops, sums = [], []
    for r in range(n_shards):
        t0, t1 = shard.trial_range(T, n_shards, r)
        a, b = shard_list(y[:, t0:t1], k)
        tops.append(a)
        sums.append(b)
    mean, pml, tvar = shard.merge(np.stack(tops), np.stack(sums), T, probs)
    om, op, ot = oracle.metrics(y, probs)
    np.testing.assert_array_equal(pml, op)
    np.testing.assert_allclose(tvar, ot, rtol=1e-12)
    np.testing.assert_allclose(mean, om, rtol=1e-12)


def test_trial_ranges_cover_every_trial_once():
    for T in (1, 7, 1000, 1_000_003):
        for world in (1, 2, 3, 8):
            ranges = [shard.trial_range(T, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == T
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1


def test_tail_count_is_the_oracle_rank():
    for n in (1, 3, 100, 10_000, 1_000_000, 999_983):
        for p in (0.5, 0.9, 0.99, 0.996, 0.999, 0.999999):
            assert shard.tail_count(p, n) == oracle.tail_count(p, n)


def test_merge_rejects_lists_shorter_than_a_probability_needs():
    from paper_1308_2572_gb300 import art
    y = _ylt()
    T = y.shape[1]
    top, sums = shard_list(y, 10)
    with pytest.raises(art.ArtError):
        shard.merge(top[None], sums[None], T, [0.99])  # needs k = 31

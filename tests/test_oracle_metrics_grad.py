"""Pins for the oracle's metrics (PML, TVaR, mean) and analytic gradients."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1308_2572_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_metrics_hand_example():
    g = json.load(open(os.path.join(GOLDEN, "metrics_example.json")))
    y = np.array(g["ylt"], dtype=np.float64)
    mean, pml, tvar = oracle.metrics(y, g["probs"])
    np.testing.assert_array_equal(mean, g["mean"])
    np.testing.assert_array_equal(pml, g["pml"])
    np.testing.assert_allclose(tvar, g["tvar"], rtol=1e-15)
    for p, k in zip(g["probs"], g["k"]):
        assert oracle.tail_count(p, y.shape[1]) == k


def test_tail_count_printed_cases():
    g = json.load(open(os.path.join(GOLDEN, "metrics_example.json")))
    for p, n, k in g["tail_count_cases"]:
        assert oracle.tail_count(p, n) == k, (p, n)


@pytest.mark.parametrize("seed", [0, 1])
def test_metrics_against_full_sort(seed):
    """PML / TVaR / mean against numpy's sort on random tables with ties."""
    rng = np.random.default_rng(seed)
    y = np.round(rng.lognormal(3, 1, size=(4, 5000)), 1)
    y[1, :2000] = 0.0
    y[2, :] = 7.0
    probs = [0.9, 0.99, 0.996, 0.999]
    mean, pml, tvar = oracle.metrics(y, probs)
    for j in range(y.shape[0]):
        s = np.sort(y[j])[::-1]
        assert mean[j] == pytest.approx(y[j].mean(), rel=1e-13)
        for q, p in enumerate(probs):
            k = oracle.tail_count(p, y.shape[1])
            assert k == int(np.ceil(round((1 - p) * y.shape[1], 6)))
            assert pml[j, q] == s[k - 1]
            assert tvar[j, q] == pytest.approx(s[:k].mean(), rel=1e-13)


def _fd_problem(seed):
    w = workloads.random_case(seed, catalogue=41, n_elt=4, n_layers=3, n_trials=25, min_len=5, max_len=40,
                              mult_range=(0.7, 1.4))
    return w.oracle_problem()


@pytest.mark.parametrize("seed", [21, 22])
def test_gradient_against_central_differences(seed):
    """Y is piecewise linear in every term, so on trials whose branch pattern
    is the same at theta - h, theta and theta + h the central difference
    equals the analytic gradient up to FP64 rounding."""
    p = _fd_problem(seed)
    L = len(p["occ_ret"])
    T = len(p["trial_off"]) - 1
    n_elt = len(p["elt_mult"])
    ones = np.ones((L, T))
    _, _, rows, pat0 = oracle.grad(p, ones, want_per_trial=True, want_pattern=True)
    checked = 0
    params = [("occ_ret", j, 0) for j in range(L)] + [("occ_lim", j, 1) for j in range(L)] + \
             [("agg_ret", j, 2) for j in range(L)] + [("agg_lim", j, 3) for j in range(L)] + \
             [("elt_mult", e, None) for e in range(n_elt)]
    for key, idx, col in params:
        h = 1e-4 * abs(p[key][idx])
        pp, pm = dict(p), dict(p)
        pp[key] = p[key].copy(); pp[key][idx] += h
        pm[key] = p[key].copy(); pm[key][idx] -= h
        yp, _, _ = oracle.ylt(pp)
        ym, _, _ = oracle.ylt(pm)
        _, _, _, patp = oracle.grad(pp, ones, want_pattern=True)
        _, _, _, patm = oracle.grad(pm, ones, want_pattern=True)
        same = (patp == pat0) & (patm == pat0)
        fd = (yp - ym) / (2 * h)
        c = col if col is not None else 4 + idx
        for j in range(L):
            if key != "elt_mult" and j != idx:
                continue
            for t in range(T):
                if not same[j, t]:
                    continue
                assert fd[j, t] == pytest.approx(rows[j, t, c], rel=1e-6, abs=1e-6 * max(1.0, abs(fd[j, t]))), (key, idx, j, t)
                checked += 1
    assert checked > 100


def test_weighted_gradient_is_sum_of_rows():
    p = _fd_problem(23)
    L = len(p["occ_ret"])
    T = len(p["trial_off"]) - 1
    g = np.random.default_rng(3).uniform(-1, 1, size=(L, T))
    gt, gm, rows, _ = oracle.grad(p, g, want_per_trial=True)
    np.testing.assert_allclose(gt, np.einsum("jt,jtq->jq", g, rows[:, :, :4]), rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(gm, np.einsum("jt,jte->e", g, rows[:, :, 4:]), rtol=1e-12, atol=1e-9)

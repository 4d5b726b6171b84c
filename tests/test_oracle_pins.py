"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a
hand-worked example (tests/golden), the closed forms of the XL terms,
identity terms that reduce the method to a plain gathered sum, invariants
that hold for any input, and brute force against the exact rational
transcription of Algorithm 1.
"""
import itertools
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.literal import algorithm1_trial
from paper_1308_2572_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _worked_problem(agg_lim, mult=(1.0, 1.0)):
    g = json.load(open(os.path.join(GOLDEN, "worked_example.json")))
    C = g["catalogue_size"]
    names = list(g["elts"])
    tab = np.zeros((len(names), C), dtype=np.float32)
    for i, n in enumerate(names):
        for ev, loss in g["elts"][n]["losses"].items():
            tab[i, int(ev)] = loss
    lim = [np.inf if g["elts"][n]["Lim"] is None else g["elts"][n]["Lim"] for n in names]
    lay = g["layer"]
    p = dict(catalogue_size=C, elt_losses=tab, elt_mult=np.array(mult, dtype=np.float64),
             elt_ded=np.array([g["elts"][n]["D"] for n in names], dtype=np.float64),
             elt_lim=np.array(lim, dtype=np.float64), layer_elt_off=np.array([0, 2], np.int32),
             layer_elt_ids=np.array([0, 1], np.int32), occ_ret=np.array([lay["OccR"]], np.float64),
             occ_lim=np.array([lay["OccL"]], np.float64), agg_ret=np.array([lay["AggR"]], np.float64),
             agg_lim=np.array([agg_lim], np.float64), event_ids=np.array(g["trial"], np.int32),
             events_per_trial=len(g["trial"]), n_trials=1)
    return g, p


@pytest.mark.parametrize("case", [0, 1])
def test_worked_example(case):
    g0, _ = _worked_problem(0)
    c = g0["cases"][case]
    _, p = _worked_problem(c["AggL"])
    y, gross, s = oracle.ylt(p, want_sum=True)
    assert y[0, 0] == c["Y"]
    assert gross[0, 0] == c["gross"]
    assert s[0, 0] == c["cumulative"][-1]
    lr, pay = oracle.ylt_running(p, want_payouts=True)
    assert lr[0, 0] == c["Y"]
    assert list(pay[0]) == c["payouts"]
    gt, gm, _, _ = oracle.grad(p, np.ones((1, 1)))
    exp = c["grad"]
    assert list(gt[0]) == [exp["OccR"], exp["OccL"], exp["AggR"], exp["AggL"]]
    assert list(gm) == [exp["m_A"], exp["m_B"]]


def test_worked_example_literal_transcription():
    """The exact transcription reproduces the hand-worked values too."""
    g, _ = _worked_problem(0)
    tables = {n: {int(k): v for k, v in g["elts"][n]["losses"].items()} for n in g["elts"]}
    terms = {n: (g["elts"][n]["m"], g["elts"][n]["D"], g["elts"][n]["Lim"]) for n in g["elts"]}
    lay = g["layer"]
    for c in g["cases"]:
        lr, pay = algorithm1_trial(g["trial"], lay["elts"], tables, terms,
                                   (lay["OccR"], lay["OccL"], lay["AggR"], c["AggL"]))
        assert lr == c["Y"] and pay == c["payouts"]


def _single(loss, m, D, Lim, occ_r, occ_l, agg_r, agg_l, repeats=1):
    p = dict(catalogue_size=1, elt_losses=np.array([[loss]], np.float32), elt_mult=np.array([m], float),
             elt_ded=np.array([D], float), elt_lim=np.array([Lim], float),
             layer_elt_off=np.array([0, 1], np.int32), layer_elt_ids=np.array([0], np.int32),
             occ_ret=np.array([occ_r], float), occ_lim=np.array([occ_l], float),
             agg_ret=np.array([agg_r], float), agg_lim=np.array([agg_l], float),
             event_ids=np.zeros(repeats, np.int32), events_per_trial=repeats, n_trials=1)
    return oracle.ylt(p)[0][0, 0]


@pytest.mark.parametrize("loss,expect", [(0, 0), (5, 0), (10, 0), (11, 1), (60, 50), (110, 100), (111, 100), (1e6, 100)])
def test_financial_terms_closed_form(loss, expect):
    """F(y) = min(max(y - D, 0), Lim) with D = 10, Lim = 100, and identity
    occurrence/aggregate terms: zero below the deductible, capped at the limit."""
    assert _single(loss, 1.0, 10.0, 100.0, 0.0, np.inf, 0.0, np.inf) == expect


@pytest.mark.parametrize("loss,expect", [(0, 0), (40, 0), (50, 0), (51, 1), (120, 70), (150, 100), (151, 100), (1e9, 100)])
def test_occurrence_terms_closed_form(loss, expect):
    """O(x) = min(max(x - OccR, 0), OccL) with OccR = 50, OccL = 100."""
    assert _single(loss, 1.0, 0.0, np.inf, 50.0, 100.0, 0.0, np.inf) == expect


@pytest.mark.parametrize("repeats,expect", [(1, 0), (3, 0), (4, 0), (5, 10), (10, 60), (12, 70), (20, 70)])
def test_aggregate_terms_closed_form(repeats, expect):
    """A(S) = min(max(S - AggR, 0), AggL) with one event of loss 10 repeated:
    S = 10 n, AggR = 40, AggL = 70; every repeat counts (indexing by position)."""
    assert _single(10.0, 1.0, 0.0, np.inf, 0.0, np.inf, 40.0, 70.0, repeats) == expect


def test_multiplier_scales_before_terms():
    """m multiplies the loss before the deductible: F(20) at m = 3, D = 10 is 50."""
    assert _single(20.0, 3.0, 10.0, np.inf, 0.0, np.inf, 0.0, np.inf) == 50.0


def _identity(w):
    p = w.oracle_problem()
    L, E = w.portfolio.n_layers, w.portfolio.n_elt
    p.update(elt_ded=np.zeros(E), elt_lim=np.full(E, np.inf), occ_ret=np.zeros(L), occ_lim=np.full(L, np.inf),
             agg_ret=np.zeros(L), agg_lim=np.full(L, np.inf))
    return p


def test_identity_terms_give_plain_gathered_sum():
    """With every retention 0 and every limit infinite, Y is the plain sum of
    m_e l_e[E_d] over the layer's ELTs and the trial's events, computed here
    by numpy fancy indexing with no reference to the method's loops."""
    w = workloads.random_case(11, catalogue=53, n_elt=6, n_layers=4, n_trials=29, mult_range=(0.5, 2.0))
    p = _identity(w)
    y, gross, _ = oracle.ylt(p)
    port, yet = w.portfolio, w.yet
    off = yet.offsets()
    for j in range(port.n_layers):
        elts = port.layer_elt_ids[port.layer_elt_off[j]:port.layer_elt_off[j + 1]]
        weighted = port.elt_losses[elts].astype(np.float64) * port.elt_mult[elts, None].astype(np.float64)
        per_event = weighted.sum(axis=0)
        for t in range(yet.n_trials):
            expect = per_event[yet.event_ids[off[t]:off[t + 1]]].sum()
            assert y[j, t] == pytest.approx(expect, rel=1e-12, abs=1e-9)
            assert gross[j, t] == pytest.approx(expect, rel=1e-12, abs=1e-9)


def test_single_elt_single_event_reduces_to_composition():
    """One ELT, one event: Y = A(O(F(l))) with the three forms nested."""
    for loss in [0.0, 3.0, 17.0, 250.0, 4000.0]:
        f = min(max(2.0 * loss - 5.0, 0.0), 300.0)
        o = min(max(f - 7.0, 0.0), 200.0)
        a = min(max(o - 11.0, 0.0), 150.0)
        assert _single(loss, 2.0, 5.0, 300.0, 7.0, 200.0, 11.0, 150.0) == a


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_invariants(seed):
    w = workloads.random_case(seed, inf_limits=(seed == 3))
    p = w.oracle_problem()
    y, gross, s = oracle.ylt(p, want_sum=True)
    port = w.portfolio
    agg_r, agg_l = port.agg_ret[:, None], port.agg_lim[:, None]
    assert np.all(y >= 0)
    assert np.all(y <= agg_l)
    assert np.all(y <= s + 1e-9 * np.maximum(s, 1))
    assert np.all(y[s <= agg_r] == 0)
    assert np.all(s <= gross * (1 + 1e-12) + 1e-9)
    # running form equals the closed form (telescoping), up to FP64 rounding
    lr, _ = oracle.ylt_running(p)
    np.testing.assert_allclose(lr, y, rtol=1e-12, atol=1e-6)


def test_permutation_invariance():
    """The trial loss does not depend on the order of the trial's events."""
    w = workloads.random_case(5)
    p = w.oracle_problem()
    y0, _, _ = oracle.ylt(p)
    rng = np.random.default_rng(0)
    ids = p["event_ids"].copy()
    off = p["trial_off"]
    for t in range(len(off) - 1):
        ids[off[t]:off[t + 1]] = rng.permutation(ids[off[t]:off[t + 1]])
    p2 = dict(p, event_ids=ids)
    y1, _, _ = oracle.ylt(p2)
    np.testing.assert_allclose(y1, y0, rtol=1e-12, atol=1e-6)


def test_monotone_in_losses_and_multipliers():
    w = workloads.random_case(7)
    p = w.oracle_problem()
    y0, _, _ = oracle.ylt(p)
    tab = p["elt_losses"].copy()
    nz = np.argwhere(tab > 0)
    rng = np.random.default_rng(1)
    for e, i in nz[rng.choice(len(nz), 10, replace=False)]:
        t2 = tab.copy()
        t2[e, i] *= 3.0
        y1, _, _ = oracle.ylt(dict(p, elt_losses=t2))
        assert np.all(y1 >= y0 - 1e-9)
    m2 = p["elt_mult"] * 1.5
    y2, _, _ = oracle.ylt(dict(p, elt_mult=m2))
    assert np.all(y2 >= y0 - 1e-9)


def test_antitone_in_retentions():
    w = workloads.random_case(8)
    p = w.oracle_problem()
    y0, _, _ = oracle.ylt(p)
    y1, _, _ = oracle.ylt(dict(p, occ_ret=p["occ_ret"] * 1.3))
    y2, _, _ = oracle.ylt(dict(p, agg_ret=p["agg_ret"] * 1.3))
    assert np.all(y1 <= y0 + 1e-9)
    assert np.all(y2 <= y0 + 1e-9)


def test_brute_force_against_exact_transcription():
    """Every id sequence of length 0..3 over a 4-event catalogue, with small
    integer losses and terms (so FP64 is exact): the C oracle's closed form
    equals Algorithm 1 transcribed literally in exact rational arithmetic."""
    rng = np.random.default_rng(2024)
    C, E = 4, 3
    tab = rng.integers(0, 40, size=(E, C)).astype(np.float32)
    tab[tab < 10] = 0
    m = np.array([1.0, 2.0, 1.0])
    D = np.array([3.0, 0.0, 7.0])
    Lim = np.array([25.0, np.inf, 30.0])
    layers = [[0, 1, 2], [1], [0, 2]]
    lterms = [(10.0, 20.0, 5.0, 30.0), (0.0, np.inf, 15.0, 40.0), (4.0, 9.0, 0.0, np.inf)]
    seqs = [s for n in range(4) for s in itertools.product(range(C), repeat=n)]
    off = np.zeros(len(seqs) + 1, np.int64)
    off[1:] = np.cumsum([len(s) for s in seqs])
    ids = np.array([e for s in seqs for e in s], dtype=np.int32)
    loff = np.array([0, 3, 4, 6], np.int32)
    lids = np.array([e for l in layers for e in l], np.int32)
    p = dict(catalogue_size=C, elt_losses=tab, elt_mult=m, elt_ded=D, elt_lim=Lim, layer_elt_off=loff,
             layer_elt_ids=lids, occ_ret=np.array([t[0] for t in lterms]), occ_lim=np.array([t[1] for t in lterms]),
             agg_ret=np.array([t[2] for t in lterms]), agg_lim=np.array([t[3] for t in lterms]),
             event_ids=ids, trial_off=off)
    y, _, _ = oracle.ylt(p)
    lr, pay = oracle.ylt_running(p, want_payouts=True)
    tables = [{i: int(tab[e, i]) for i in range(C) if tab[e, i]} for e in range(E)]
    inf2none = lambda v: None if np.isinf(v) else Fraction(int(v))
    terms = [(Fraction(int(m[e])), Fraction(int(D[e])), inf2none(Lim[e])) for e in range(E)]
    assert len(seqs) == 4 ** 3 + 4 ** 2 + 4 + 1
    for j, layer in enumerate(layers):
        lt = (Fraction(int(lterms[j][0])), inf2none(lterms[j][1]), Fraction(int(lterms[j][2])), inf2none(lterms[j][3]))
        for t, s in enumerate(seqs):
            exact, exact_pay = algorithm1_trial(list(s), layer, tables, terms, lt)
            assert y[j, t] == exact
            assert lr[j, t] == exact
            assert list(pay[j, off[t]:off[t + 1]]) == [float(v) for v in exact_pay]

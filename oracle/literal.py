"""Algorithm 1 of the paper, step by step, in exact rational arithmetic.

TEST INFRASTRUCTURE ONLY (tiny inputs; pure-Python loops). It is the
brute-force pin for the C oracle: every value is a ``fractions.Fraction``,
so no rounding can hide a dropped term or a wrong index.

It follows the algorithm's loops in order for one layer and one trial:
  per ELT of the layer: look up the loss of every event of the trial
  (step 1), apply that ELT's financial terms (step 2) and accumulate into
  the per-event loss lo_d; then the occurrence terms on every lo_d
  (step 3); the cumulative sum over the trial; the aggregate terms on every
  cumulative value (step 4); the per-event difference against the previous
  cumulative value (nothing is paid before the first event); and the trial
  loss lr as the sum of those differences.

Readings (the paper is silent or garbled here): financial terms of an ELT
are F(y) = min(max(m*y - D, 0), Lim); lo is indexed by trial position; the
difference uses the un-overwritten cumulative values.
"""
from __future__ import annotations

from fractions import Fraction
from typing import Sequence


def _xl(v, ret, lim):
    """min(max(v - ret, 0), lim); lim may be None for an unlimited cover."""
    w = v - ret
    if w < 0:
        w = Fraction(0)
    if lim is not None and w > lim:
        w = lim
    return w


def algorithm1_trial(trial_events: Sequence[int], layer_elts: Sequence[int], elt_tables,
                     elt_terms, layer_terms):
    """Trial loss lr and per-event payouts for one layer.

    elt_tables[e] maps an event id to its loss (absent ids have loss 0);
    elt_terms[e] = (m, D, Lim); layer_terms = (OccR, OccL, AggR, AggL);
    Lim, OccL and AggL may be None (unlimited). Values should be Fractions
    or ints.
    """
    k = len(trial_events)
    lo = [Fraction(0)] * k
    for c in layer_elts:
        table = elt_tables[c]
        m, D, Lim = elt_terms[c]
        x = [Fraction(table.get(ev, 0)) for ev in trial_events]            # step 1
        l = [_xl(Fraction(m) * xd, Fraction(D), None if Lim is None else Fraction(Lim)) for xd in x]  # step 2
        lo = [lo[d] + l[d] for d in range(k)]                               # accumulate
    occ_r, occ_l, agg_r, agg_l = layer_terms
    occ_l = None if occ_l is None else Fraction(occ_l)
    agg_l = None if agg_l is None else Fraction(agg_l)
    lo = [_xl(v, Fraction(occ_r), occ_l) for v in lo]                       # step 3
    cum, run = [], Fraction(0)
    for v in lo:                                                            # cumulative sum
        run += v
        cum.append(run)
    capped = [_xl(v, Fraction(agg_r), agg_l) for v in cum]                  # step 4
    payouts = [capped[d] - (capped[d - 1] if d else Fraction(0)) for d in range(k)]  # difference
    lr = Fraction(0)
    for p in payouts:                                                       # trial loss
        lr += p
    return lr, payouts

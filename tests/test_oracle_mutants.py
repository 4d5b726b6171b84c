"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of ara_oracle.c (a dropped term, a
wrong sign, a transposed index, a wrong term, an off-by-one), compiles it on
the CPU and runs the pin suites against it; at least one pin must fail.
"""
import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ara_oracle.c")
PINS = [os.path.join(ROOT, "tests", "test_oracle_pins.py"), os.path.join(ROOT, "tests", "test_oracle_metrics_grad.py")]

MUTANTS = {
    "dropped_multiplier": ("x += xl(p->elt_mult[e] * y, p->elt_ded[e], p->elt_lim[e]);",
                           "x += xl(y, p->elt_ded[e], p->elt_lim[e]);"),
    "no_elt_accumulation": ("x += xl(p->elt_mult[e] * y, p->elt_ded[e], p->elt_lim[e]);",
                            "x = xl(p->elt_mult[e] * y, p->elt_ded[e], p->elt_lim[e]);"),
    "retention_sign": ("double w = v - ret;\n    if (w < 0.0) w = 0.0;", "double w = v + ret;\n    if (w < 0.0) w = 0.0;"),
    "dropped_cap": ("if (w > lim) w = lim;\n    return w;", "return w;"),
    "occurrence_uses_agg_limit": ("s += xl(x, p->occ_ret[j], p->occ_lim[j]);", "s += xl(x, p->occ_ret[j], p->agg_lim[j]);"),
    "aggregate_terms_dropped": ("ylt[w] = xl(s, p->agg_ret[j], p->agg_lim[j]);", "ylt[w] = s;"),
    "transposed_table_index": ("double y = (double)p->elt_losses[(int64_t)e * p->catalogue_size + id];",
                               "double y = (double)p->elt_losses[(int64_t)id * p->n_elt + e];"),
    "tail_count_floor": ("(int64_t)ceil(q);", "(int64_t)floor(q);"),
    "pml_off_by_one": ("pml[(int64_t)j * n_p + q] = buf[k - 1];", "pml[(int64_t)j * n_p + q] = buf[k < n_trials ? k : k - 1];"),
    "grad_occ_sign": ("row[0] = -a * n_occ_mid;", "row[0] = a * n_occ_mid;"),
    "grad_mult_ignores_branch": ("if (xl_branch(elt_mult[e] * y, elt_ded[e], elt_lim[e]) == 1) dm[e] += y;", "dm[e] += y;"),
    "running_first_payout": ("double pd = cum[d] - (d ? cum[d - 1] : 0.0);", "double pd = cum[d] - (d ? cum[d - 1] : cum[d]);"),
    "tvar_wrong_divisor": ("tvar[(int64_t)j * n_p + q] = top / (double)k;",
                           "tvar[(int64_t)j * n_p + q] = top / (double)(k > 1 ? k - 1 : k);"),
    "tvar_drops_kth": ("for (int64_t i = 0; i < k; ++i) top += buf[i];", "for (int64_t i = 0; i + 1 < k; ++i) top += buf[i];"),
    "mean_wrong_divisor": ("mean[j] = s / (double)n_trials;", "mean[j] = s / (double)(n_trials > 1 ? n_trials - 1 : 1);"),
    "grad_occ_lim_counts_mid": ("row[1] = a * n_occ_cap;", "row[1] = a * n_occ_mid;"),
    "grad_agg_lim_on_mid_branch": ("row[3] = cc;", "row[3] = a;"),
    "grad_mult_ignores_agg_branch": ("for (int32_t e = 0; e < n_elt; ++e) dm[e] *= a;", ""),
    "aggregate_retention_dropped": ("ylt[w] = xl(s, p->agg_ret[j], p->agg_lim[j]);", "ylt[w] = xl(s, 0.0, p->agg_lim[j]);"),
    "running_occurrence_limit_dropped": ("lo[d] = xl(lo[d], occ_ret[j], occ_lim[j]);",
                                         "lo[d] = xl(lo[d], occ_ret[j], INFINITY);"),
    "running_cumulative_restarts": ("cum[d] = lo[d] + (d ? cum[d - 1] : 0.0);", "cum[d] = lo[d];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    d = tempfile.mkdtemp(prefix="ara_mutant_")
    try:
        c = os.path.join(d, "m.c")
        so = os.path.join(d, "libm.so")
        open(c, "w").write(src.replace(old, new, 1))
        subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", so, c, "-lm"], check=True)
        env = dict(os.environ, ARA_ORACLE_LIB=so, OMP_NUM_THREADS="2")
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PINS],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, f"no pin caught mutant {name}:\n{r.stdout[-2000:]}"
    finally:
        shutil.rmtree(d, ignore_errors=True)


# The exact transcription (oracle/literal.py) is a pin itself: planted
# mistakes in it must fail the worked example or the brute-force comparison
# with the C oracle.
LIT = os.path.join(ROOT, "oracle", "literal.py")
LIT_MUTANTS = {
    "no_elt_accumulation": ("lo = [lo[d] + l[d] for d in range(k)]", "lo = [l[d] for d in range(k)]"),
    "occurrence_limit_dropped": ("lo = [_xl(v, Fraction(occ_r), occ_l) for v in lo]",
                                 "lo = [_xl(v, Fraction(occ_r), None) for v in lo]"),
    "first_payout": ("(capped[d - 1] if d else Fraction(0))", "(capped[d - 1] if d else capped[0])"),
    "multiplier_dropped": ("_xl(Fraction(m) * xd,", "_xl(xd,"),
    "cumulative_restarts": ("run += v", "run = v"),
    "deductible_sign": ("w = v - ret", "w = v + ret"),
}


@pytest.mark.parametrize("name", sorted(LIT_MUTANTS))
def test_pins_catch_planted_mistake_in_the_transcription(name, monkeypatch):
    import types

    import test_oracle_pins as pins
    old, new = LIT_MUTANTS[name]
    src = open(LIT).read()
    assert src.count(old) >= 1, f"mutation site for {name} not found"
    mod = types.ModuleType("literal_mutant")
    exec(compile(src.replace(old, new, 1), "literal_mutant", "exec"), mod.__dict__)
    monkeypatch.setattr(pins, "algorithm1_trial", mod.algorithm1_trial)
    caught = []
    for pin in (pins.test_worked_example_literal_transcription, pins.test_brute_force_against_exact_transcription):
        try:
            pin()
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"no pin caught the transcription mutant {name}"


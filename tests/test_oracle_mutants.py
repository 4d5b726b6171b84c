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

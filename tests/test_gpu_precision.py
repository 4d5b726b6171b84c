"""Precision of every forward variant on the 128-layer, 512-ELT workload
(first 3,000 trials): |dY| <= 1e-6 G per output and PML / TVaR / mean
within 1e-6 relative of the FP64 oracle, for the mixed FP32/FP64 forms and
the all-FP64 forms (tests/precision_report.py prints the full report)."""
import pytest

from precision_report import report

pytestmark = pytest.mark.gpu


def test_precision_report_c4_prefix():
    r = report("c4", 3000)
    for name, v in r["variants"].items():
        assert v["max_abs_dY_over_G"] <= 1e-6, name
        assert max(v["pml_rel_err"]) <= 1e-6, name
        assert max(v["tvar_rel_err"]) <= 1e-6, name
        assert v["mean_rel_err"] <= 1e-6, name
    # the all-FP64 forms (over FP64 occurrence tables and over the FP64 pool)
    # are the more accurate ones
    for name in ("all-FP64 (occurrence tables)", "all-FP64 (FP64 pool)"):
        fp64 = r["variants"][name]["max_abs_dY_over_G"]
        assert fp64 <= r["variants"]["batched (FP32 + FP64 aggregate)"]["max_abs_dY_over_G"], name
        assert fp64 <= 1e-12, name

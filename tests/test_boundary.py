"""The C-ABI library: it builds, loads without a GPU, exports every entry
point include/art.h declares, and its host-side validation rejects bad
arguments before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def art():
    from paper_1308_2572_gb300 import art as a
    from paper_1308_2572_gb300 import build
    build.build()
    a.lib()
    return a


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "art.h")).read()
    return sorted(set(re.findall(r"ART_API\s+[\w\s\*]+?\b(art_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for n in ["art_create_portfolio", "art_run_ylt", "art_metrics", "art_run_ylt_backward", "art_destroy_portfolio",
              "art_status_string", "art_get_device_status"]:
        assert n in names


def test_every_entry_point_is_documented():
    """Each declaration in include/art.h follows a comment that cites the
    paper's passage (or says the paper has no counterpart) and states the
    errors it returns (or that it never fails)."""
    src = open(os.path.join(ROOT, "include", "art.h")).read()
    for m in re.finditer(r"ART_API\s+[\w\s\*]+?\b(art_\w+)\s*\(", src):
        before = src[:m.start()]
        end = before.rfind("*/")
        block = before[before.rfind("/*", 0, end):end]
        assert re.search(r"Section|Algorithm|paper", block), m.group(1)
        assert re.search(r"Errors|ART_E|never fails|no-op", block), m.group(1)


def test_library_exports_every_declared_symbol(art):
    L = art.lib()
    names = declared_entry_points()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(art.EXPORTS) == names


def test_status_strings(art):
    for code in range(7):
        s = art.art_status_string(code)
        assert s.startswith("ART_")
    assert art.art_status_string(99) == "unknown art_status"
    assert art.art_version() >= 10000


def test_create_rejects_bad_arguments_on_the_host(art):
    L = art.lib()
    out = ctypes.c_void_p()
    off = np.array([0, 2], np.int32)
    ids = np.array([0, 1], np.int32)
    ded = np.zeros(2, np.float32)
    lim = np.full(2, np.inf, np.float32)
    terms = (art.LayerTerms * 1)(art.LayerTerms(0.0, np.inf, 0.0, np.inf))
    fake = ctypes.c_void_p(16)  # never dereferenced: validation fails first

    def call(C=10, n_elt=2, losses=fake, off_=off, ids_=ids, ded_=ded, lim_=lim, n_layers=1, out_=ctypes.byref(out)):
        return L.art_create_portfolio(C, n_elt, losses, None, ded_.ctypes.data, lim_.ctypes.data, n_layers,
                                      off_.ctypes.data, ids_.ctypes.data, ctypes.cast(terms, ctypes.c_void_p), None,
                                      None, out_)

    assert call(out_=None) == art.ART_EINVAL
    assert call(C=0) == art.ART_EINVAL
    assert call(n_elt=0) == art.ART_EINVAL
    assert call(n_layers=0) == art.ART_EINVAL
    assert call(losses=None) == art.ART_EINVAL
    assert call(off_=np.array([1, 2], np.int32)) == art.ART_EINVAL          # does not start at 0
    assert call(off_=np.array([0, 0], np.int32)) == art.ART_EINVAL          # empty layer
    assert call(ids_=np.array([0, 2], np.int32)) == art.ART_EINVAL          # ELT id out of range
    assert call(ids_=np.array([1, 1], np.int32)) == art.ART_EINVAL          # duplicate ELT in a layer
    assert call(off_=np.array([0, 33], np.int32), ids_=np.arange(33, dtype=np.int32), n_elt=40,
                ded_=np.zeros(40, np.float32), lim_=np.ones(40, np.float32)) == art.ART_EINVAL  # > 32 ELTs
    assert call(ded_=np.array([-1, 0], np.float32)) == art.ART_EINVAL       # negative deductible
    assert call(ded_=np.array([np.nan, 0], np.float32)) == art.ART_EINVAL
    assert call(lim_=np.array([0, 1], np.float32)) == art.ART_EINVAL        # zero limit


def test_other_entry_points_reject_bad_arguments_on_the_host(art):
    L = art.lib()
    probs = np.array([0.99])
    fake = ctypes.c_void_p(16)
    assert L.art_run_ylt(None, 10, fake, None, 5, fake, None, None) == art.ART_EINVAL
    assert L.art_run_ylt_host(None, 10, fake, None, 5, fake, None) == art.ART_EINVAL
    assert L.art_run_ylt_host_metrics(None, 10, fake, None, 5, None, probs.ctypes.data, 1, None, None, None,
                                      None) == art.ART_EINVAL
    assert L.art_metrics(None, 10, 1, probs.ctypes.data, 1, None, None, None, None) == art.ART_EINVAL
    assert L.art_metrics(fake, 0, 1, probs.ctypes.data, 1, None, None, None, None) == art.ART_EINVAL
    bad = np.array([1.0])
    assert L.art_metrics(fake, 10, 1, bad.ctypes.data, 1, None, None, None, None) == art.ART_EINVAL
    assert L.art_metrics(fake, 10, 1, probs.ctypes.data, 9, None, None, None, None) == art.ART_EINVAL
    # the documented size limits: trials below 2^31, layers up to 65535
    assert L.art_metrics(fake, 1 << 31, 1, probs.ctypes.data, 1, None, None, None, None) == art.ART_EINVAL
    assert L.art_metrics(fake, 10, 65536, probs.ctypes.data, 1, None, None, None, None) == art.ART_EINVAL
    assert L.art_metrics(fake, 10, 0, probs.ctypes.data, 1, None, None, None, None) == art.ART_EINVAL
    assert L.art_metrics_noalloc(fake, 10, 65536, probs.ctypes.data, 1, None, None, None, None) == art.ART_EINVAL
    # TVaR gradients need the PML and the probabilities
    assert L.art_metrics_backward(fake, 10, 1, None, 0, None, None, fake, fake, None) == art.ART_EINVAL
    assert L.art_metrics_backward(fake, 10, 1, probs.ctypes.data, 1, None, None, fake, fake, None) == art.ART_EINVAL
    assert L.art_metrics_backward(fake, 10, 1, None, 0, None, None, fake, None, None) == art.ART_EINVAL
    assert L.art_run_ylt_backward(None, 10, fake, None, 5, fake, fake, fake, fake, None) == art.ART_EINVAL
    assert L.art_get_device_status(None, None) == art.ART_EINVAL
    assert L.art_run_payouts(None, 0, 10, fake, None, 5, None, None, None, None) == art.ART_EINVAL
    assert L.art_update_terms(None, None, None, None, None) == art.ART_EINVAL
    assert L.art_set_variant(None, 1, 0, 0) == art.ART_EINVAL
    assert L.art_set_flags(None, 0) == art.ART_EINVAL
    assert L.art_get_footprint(None, None, None, None, None, None) == art.ART_EINVAL
    out = ctypes.c_double()
    assert L.art_probe(99, 1 << 20, 1, ctypes.byref(out)) == art.ART_EINVAL
    assert L.art_probe(0, 16, 1, ctypes.byref(out)) == art.ART_EINVAL
    assert L.art_probe(0, 1 << 20, 0, ctypes.byref(out)) == art.ART_EINVAL
    L.art_destroy_portfolio(None)  # no-op


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    from paper_1308_2572_gb300 import art as a
    monkeypatch.setattr(a, "_lib", None)
    monkeypatch.setattr(a, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        a.lib()

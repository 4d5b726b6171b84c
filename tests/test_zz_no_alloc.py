"""art_metrics_noalloc against art_metrics and against the FP64 oracle.

art_metrics_noalloc serves callers that cannot allocate device memory while
they run (a fixed memory budget reserved at start-up, a device allocator
owned by another framework, latency-critical paths): it computes the same
mean, PML and TVaR over the library's fixed static scratch instead of the
stream-ordered allocator. This file is collected last on purpose, so that a
run stopping at its first failure has run every other test first; it also
passes alone in a fresh process.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1308_2572_gb300 import art

pytestmark = pytest.mark.gpu


def _tables():
    g = torch.Generator(device="cpu").manual_seed(7)
    a = torch.distributions.LogNormal(10.0, 2.0).sample((5, 100_003)).double()
    a[1, :40_000] = 0.0                       # many zero trials
    a[2] = torch.round(a[2] / 1e5) * 1e5      # heavy ties
    a[3] = 4.0e7                              # every trial capped at the same value
    b = torch.rand((3, 77_777), generator=g, dtype=torch.float64) * 1e8
    return [(a.cuda(), [0.9, 0.99, 0.996, 0.999]), (b.cuda(), [0.5, 0.99])]


def _run(fn, ylt, probs):
    L, T = ylt.shape
    mean = torch.full((L,), -1.0, dtype=torch.float64, device="cuda")
    pml = torch.full((L, len(probs)), -1.0, dtype=torch.float64, device="cuda")
    tvar = torch.full((L, len(probs)), -1.0, dtype=torch.float64, device="cuda")
    fn(ylt, T, L, probs, mean, pml, tvar)
    torch.cuda.synchronize()
    return mean.cpu().numpy(), pml.cpu().numpy(), tvar.cpu().numpy()


def test_noalloc_metrics_match_allocating_entry_point_on_two_calls_in_a_row():
    art.lib()
    tables = _tables()
    expect = [_run(art.art_metrics, y, p) for y, p in tables]
    # two calls in a row on different tables, then the first table again: a
    # scratch left dirty by the previous call would show here
    for (y, p), ref in [(tables[0], expect[0]), (tables[1], expect[1]), (tables[0], expect[0])]:
        got = _run(art.art_metrics_noalloc, y, p)
        np.testing.assert_array_equal(got[1], ref[1])            # the k-th largest is selected exactly
        np.testing.assert_allclose(got[2], ref[2], rtol=1e-12)    # TVaR
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-12)    # mean
        # and against the oracle's full sort of the same table
        om, op, ot = oracle.metrics(y.cpu().numpy(), p)
        np.testing.assert_array_equal(got[1], op)
        np.testing.assert_allclose(got[2], ot, rtol=1e-12)
        np.testing.assert_allclose(got[0], om, rtol=1e-12)


def test_noalloc_metrics_reject_requests_beyond_the_static_scratch():
    art.lib()
    ylt = torch.zeros((2000, 8), dtype=torch.float64, device="cuda")
    probs = [0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8]
    with pytest.raises(art.ArtError, match="static scratch"):
        _run(art.art_metrics_noalloc, ylt, probs)
    # a request that fits still works afterwards
    y, p = _tables()[1]
    ref = _run(art.art_metrics, y, p)
    got = _run(art.art_metrics_noalloc, y, p)
    np.testing.assert_array_equal(got[1], ref[1])

"""Algorithm 1's running form on the GPU (art_run_payouts) against the
oracle's running form: per-event payouts p_d = A(C_d) - A(C_{d-1}), the
event that exhausts the aggregate limit, and the trial loss."""
import numpy as np
import pytest
import torch

import oracle
from paper_1308_2572_gb300 import art, workloads

from gpu_util import device_yet

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["ragged", "dense", "inf_limits", "c0u"])
def test_payouts_match_oracle_running_form(case):
    if case == "c0u":
        w = workloads.make("c0u", n_trials=1500)
    else:
        kw = {"ragged": dict(seed=401, n_trials=400, min_len=0, max_len=150),
              "dense": dict(seed=402, n_trials=300, dense_k=64),
              "inf_limits": dict(seed=403, n_trials=300, inf_limits=True)}[case]
        w = workloads.random_case(**kw)
    prob = w.oracle_problem()
    lr_ref, pay_ref = oracle.ylt_running(prob, want_payouts=True)
    _, gross, _ = oracle.ylt(prob)
    off = w.yet.offsets()
    p = art.portfolio_from_workload(w)
    try:
        ids, doff, k, T = device_yet(w)
        for j in range(w.portfolio.n_layers):
            pay = torch.full((w.yet.n_events,), -7.0, dtype=torch.float64, device="cuda")
            ex = torch.full((T,), -9, dtype=torch.int32, device="cuda")
            yl = torch.full((T,), -1.0, dtype=torch.float64, device="cuda")
            art.art_run_payouts(p, j, T, ids, doff, k, pay, ex, yl)
            torch.cuda.synchronize()
            assert art.art_get_device_status(p) == art.ART_OK
            pay, ex, yl = pay.cpu().numpy(), ex.cpu().numpy(), yl.cpu().numpy()
            g_event = np.repeat(gross[j], np.diff(off))  # each event's tolerance base: its trial's gross loss
            assert np.all(np.abs(pay - pay_ref[j]) <= 1e-6 * g_event + 1e-9), (case, j)
            assert np.all(np.abs(yl - lr_ref[j]) <= 1e-6 * gross[j] + 1e-9), (case, j)
            assert np.all(pay >= -1e-6 * g_event)  # payouts are non-negative
            agg_l = w.portfolio.agg_lim[j]
            for t in range(T):
                cum = np.cumsum(pay_ref[j, off[t]:off[t + 1]])
                if ex[t] < 0:
                    assert not np.isfinite(agg_l) or cum.size == 0 or cum[-1] < agg_l * (1 + 1e-9) + 1e-6 * gross[j, t]
                else:
                    d = ex[t]
                    tol = 1e-6 * gross[j, t] + 1e-9 * agg_l
                    assert cum[d] >= agg_l - tol
                    assert d == 0 or cum[d - 1] <= agg_l + tol
    finally:
        p.close()

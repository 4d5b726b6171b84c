"""``torch.autograd.Function`` around the forward and adjoint kernels.

The pricing sensitivity: gradients of each layer's expected loss and TVaR_p
with respect to the layer terms (OccR, OccL, AggR, AggL) and the per-ELT loss
multipliers. Forward: art_update_terms, art_run_ylt (recording the aggregate
branch of every (layer, trial)), art_metrics. Backward: art_metrics_backward
(dLoss/dYLT), then art_run_ylt_backward (the adjoint kernel, which re-reads
only trials on the middle aggregate branch). Terms are host-side FP64 tensors;
FP32 rounding of OccR, OccL and the ELT terms happens in the library.

The portfolio holds one set of terms, and the adjoint differentiates at the
terms the portfolio holds when it runs. Each forward therefore records the
terms it applied (as rounded by the library), and its backward re-applies
them when the portfolio has moved on -- another forward in between, a
finite-difference evaluation, a second scenario -- runs the adjoint, waits
for it and puts the portfolio's terms back as it found them.
"""
from __future__ import annotations

import numpy as np
import torch

from . import art


def _same_terms(a, b) -> bool:
    return all(np.array_equal(x, y) for x, y in zip(a, b))


class ARAFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, portfolio, yet, probs, occ_ret, occ_lim, agg_ret, agg_lim, elt_mult):
        """yet = (event_ids CUDA int32, trial_off CUDA int64 or None, K, n_trials).
        Returns (mean [L], tvar [L][n_p]) as CPU float64 tensors."""
        ids, off, k, n_trials = yet
        L = portfolio.n_layers
        terms = torch.stack([occ_ret, occ_lim, agg_ret, agg_lim], dim=1).detach().cpu().numpy()
        art.art_update_terms(portfolio, elt_mult=elt_mult.detach().cpu().numpy(), terms=terms)
        dev = ids.device
        ylt = torch.empty((L, n_trials), dtype=torch.float64, device=dev)
        branch = torch.empty((L, n_trials), dtype=torch.uint8, device=dev)
        art.art_run_ylt(portfolio, n_trials, ids, off, k, ylt, branch)
        n_p = len(probs)
        mean = torch.empty(L, dtype=torch.float64, device=dev)
        pml = torch.empty((L, n_p), dtype=torch.float64, device=dev)
        tvar = torch.empty((L, n_p), dtype=torch.float64, device=dev)
        art.art_metrics(ylt, n_trials, L, probs, mean, pml, tvar)
        ctx.portfolio, ctx.yet, ctx.probs = portfolio, yet, np.asarray(probs, dtype=np.float64)
        # the terms as the kernels applied them (after FP32 rounding)
        ctx.terms_applied = art.art_get_terms(portfolio)
        ctx.save_for_backward(ylt, branch, pml)
        return mean.cpu(), tvar.cpu()

    @staticmethod
    def backward(ctx, g_mean, g_tvar):
        ylt, branch, pml = ctx.saved_tensors
        ids, off, k, n_trials = ctx.yet
        p = ctx.portfolio
        L = p.n_layers
        dev = ylt.device
        gm = g_mean.to(dev, torch.float64).contiguous() if g_mean is not None else torch.zeros(L, dtype=torch.float64, device=dev)
        gt = g_tvar.to(dev, torch.float64).contiguous() if g_tvar is not None else None
        grad_ylt = torch.empty_like(ylt)
        art.art_metrics_backward(ylt, n_trials, L, ctx.probs, pml, gm, gt, grad_ylt)
        grad_terms = torch.empty((L, 4), dtype=torch.float64, device=dev)
        grad_mult = torch.empty(p.n_elt, dtype=torch.float64, device=dev)
        current = art.art_get_terms(p)
        moved = not _same_terms(current, ctx.terms_applied)
        if moved:
            # work already queued may still read the portfolio's terms
            torch.cuda.current_stream(dev).synchronize()
            m, d, l, t = ctx.terms_applied
            art.art_update_terms(p, elt_mult=m, elt_ded=d, elt_lim=l, terms=t)
        try:
            art.art_run_ylt_backward(p, n_trials, ids, off, k, branch, grad_ylt, grad_terms, grad_mult)
        finally:
            if moved:
                # the adjoint reads the terms while it runs: wait for it before
                # giving the portfolio its terms back
                torch.cuda.current_stream(dev).synchronize()
                m, d, l, t = current
                art.art_update_terms(p, elt_mult=m, elt_ded=d, elt_lim=l, terms=t)
        gtc = grad_terms.cpu()
        return (None, None, None, gtc[:, 0], gtc[:, 1], gtc[:, 2], gtc[:, 3], grad_mult.cpu())


def layer_metrics(portfolio, yet, probs, occ_ret, occ_lim, agg_ret, agg_lim, elt_mult):
    """Differentiable (expected loss per layer, TVaR per layer and probability)."""
    return ARAFunction.apply(portfolio, yet, probs, occ_ret, occ_lim, agg_ret, agg_lim, elt_mult)

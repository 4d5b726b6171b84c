"""Plain FP64 CPU oracle for aggregate risk analysis (Section II, Algorithm 1).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's CPU
baseline call it; the product path never does. It shares no code with the
CUDA library (``paper_1308_2572_gb300``) and imports nothing from it.

The arithmetic lives in ``ara_oracle.c`` (plain C, FP64, OpenMP over
(layer, trial) pairs) and, for tiny inputs, in ``literal.py`` (exact rational
arithmetic, Algorithm 1 step by step). This module only marshals numpy arrays
into the C library, compiling it with gcc on first use when it is missing.

Parity status per function (pins live in ``tests/test_oracle_*.py``):
  ylt, ylt_running  pinned: hand-worked example, closed forms of the XL terms,
                    identity terms (plain gathered sum), invariants, brute
                    force against the exact literal transcription;
  metrics           pinned: full-sort definition on hand-built tables, k rule;
  tail_count        pinned: printed values (N=1e4, p=0.99 gives 100);
  grad              pinned: hand-worked example, central finite differences
                    on unchanged branch patterns.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ara_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libara_oracle.so")

# The compile line; __graft_entry__.build() runs the same command.
GCC_CMD = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", _LIB_PATH, _SRC, "-lm"]

_lib = None


def _compile() -> None:
    os.makedirs(_BUILD, exist_ok=True)
    subprocess.run(GCC_CMD, check=True)


def _load():
    global _lib
    if _lib is not None:
        return _lib
    # ARA_ORACLE_LIB points the wrappers at another build of ara_oracle.c;
    # the mutation test uses it to check that the pins catch planted mistakes.
    path = os.environ.get("ARA_ORACLE_LIB")
    if path is None:
        path = _LIB_PATH
        if not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
            _compile()
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    common = [i32, i32, P, P, P, P, i32, P, P, P, P, P, P, P, P, i32, i64, P, i64]
    lib.ara_oracle_ylt.argtypes = common + [P, P, P]
    lib.ara_oracle_ylt.restype = ctypes.c_int
    lib.ara_oracle_ylt_running.argtypes = common + [P, P]
    lib.ara_oracle_ylt_running.restype = ctypes.c_int
    lib.ara_oracle_grad.argtypes = common + [P, P, P, P, P]
    lib.ara_oracle_grad.restype = ctypes.c_int
    lib.ara_oracle_metrics.argtypes = [P, i64, i32, P, i32, P, P, P]
    lib.ara_oracle_metrics.restype = ctypes.c_int
    lib.ara_oracle_tail_count.argtypes = [ctypes.c_double, i64]
    lib.ara_oracle_tail_count.restype = i64
    lib.ara_oracle_num_threads.argtypes = []
    lib.ara_oracle_num_threads.restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    pass


def _common_args(p, trials):
    """Validate and convert one problem description (a dict) to C arguments.

    Keys: catalogue_size, elt_losses [n_elt][C] float32, elt_mult/elt_ded/
    elt_lim [n_elt] (float64), layer_elt_off [L+1] int32, layer_elt_ids int32,
    occ_ret/occ_lim/agg_ret/agg_lim [L] float64, event_ids int32, and either
    trial_off [T+1] int64 or events_per_trial with n_trials.
    """
    C = int(p["catalogue_size"])
    losses = np.ascontiguousarray(p["elt_losses"], dtype=np.float32)
    n_elt = losses.shape[0]
    f64 = lambda k: np.ascontiguousarray(p[k], dtype=np.float64)
    mult, ded, lim = f64("elt_mult"), f64("elt_ded"), f64("elt_lim")
    loff = np.ascontiguousarray(p["layer_elt_off"], dtype=np.int32)
    lids = np.ascontiguousarray(p["layer_elt_ids"], dtype=np.int32)
    n_layers = loff.shape[0] - 1
    occ_ret, occ_lim, agg_ret, agg_lim = f64("occ_ret"), f64("occ_lim"), f64("agg_ret"), f64("agg_lim")
    ids = np.ascontiguousarray(p["event_ids"], dtype=np.int32).reshape(-1)
    toff = p.get("trial_off")
    if toff is not None:
        toff = np.ascontiguousarray(toff, dtype=np.int64)
        n_trials = toff.shape[0] - 1
        K = 0
    else:
        K = int(p["events_per_trial"])
        n_trials = int(p["n_trials"])
    if trials is not None:
        trials = np.ascontiguousarray(trials, dtype=np.int64)
        n_out = trials.shape[0]
    else:
        n_out = n_trials
    keep = (losses, mult, ded, lim, loff, lids, occ_ret, occ_lim, agg_ret, agg_lim, ids, toff, trials)
    args = [C, n_elt, _ptr(losses), _ptr(mult), _ptr(ded), _ptr(lim), n_layers, _ptr(loff), _ptr(lids),
            _ptr(occ_ret), _ptr(occ_lim), _ptr(agg_ret), _ptr(agg_lim), _ptr(ids), _ptr(toff), K,
            n_trials, _ptr(trials), n_out]
    return args, keep, n_layers, n_out, n_elt


def ylt(p, trials=None, want_gross=True, want_sum=False):
    """Closed form Y = A(sum_d O(x_d)) per (layer, trial); Algorithm 1 steps 1-4.

    Returns (ylt, gross, agg_sum) arrays of shape [n_layers][n_out]; gross is
    the trial's gross loss sum_d sum_e m_e l_e[E_d] (the tolerance base), and
    agg_sum the occurrence-net aggregate S before the aggregate terms.
    """
    lib = _load()
    args, keep, L, n_out, _ = _common_args(p, trials)
    out = np.zeros((L, n_out), dtype=np.float64)
    gross = np.zeros((L, n_out), dtype=np.float64) if want_gross else None
    s = np.zeros((L, n_out), dtype=np.float64) if want_sum else None
    rc = lib.ara_oracle_ylt(*args, _ptr(out), _ptr(gross), _ptr(s))
    if rc:
        raise OracleError(f"ara_oracle_ylt rejected its inputs (status {rc})")
    return out, gross, s


def ylt_running(p, trials=None, want_payouts=False):
    """Algorithm 1 in its own step order (cumulative sum, aggregate terms per
    cumulative value, per-event difference, sum). Returns (lr, payouts);
    payouts is [n_layers][sum of selected trial lengths] or None."""
    lib = _load()
    args, keep, L, n_out, _ = _common_args(p, trials)
    lr = np.zeros((L, n_out), dtype=np.float64)
    payouts = None
    if want_payouts:
        toff = p.get("trial_off")
        sel = np.arange(n_out) if trials is None else np.asarray(trials)
        if toff is not None:
            toff = np.asarray(toff, dtype=np.int64)
            total = int(np.sum(toff[sel + 1] - toff[sel]))
        else:
            total = int(p["events_per_trial"]) * len(sel)
        payouts = np.zeros((L, total), dtype=np.float64)
    rc = lib.ara_oracle_ylt_running(*args, _ptr(lr), _ptr(payouts))
    if rc:
        raise OracleError(f"ara_oracle_ylt_running rejected its inputs (status {rc})")
    return lr, payouts


def grad(p, grad_ylt, trials=None, want_per_trial=False, want_pattern=False):
    """Analytic gradient of sum g_{t,j} Y_{t,j} with respect to (OccR, OccL,
    AggR, AggL) per layer and the ELT multipliers. Returns (grad_terms [L][4],
    grad_mult [n_elt], per_trial [L][n_out][4+n_elt] or None,
    pattern [L][n_out] uint64 or None)."""
    lib = _load()
    args, keep, L, n_out, n_elt = _common_args(p, trials)
    g = np.ascontiguousarray(grad_ylt, dtype=np.float64).reshape(L, n_out)
    gt = np.zeros((L, 4), dtype=np.float64)
    gm = np.zeros((n_elt,), dtype=np.float64)
    pt = np.zeros((L, n_out, 4 + n_elt), dtype=np.float64) if want_per_trial else None
    pat = np.zeros((L, n_out), dtype=np.uint64) if want_pattern else None
    rc = lib.ara_oracle_grad(*args, _ptr(g), _ptr(gt), _ptr(gm), _ptr(pt), _ptr(pat))
    if rc:
        raise OracleError(f"ara_oracle_grad rejected its inputs (status {rc})")
    return gt, gm, pt, pat


def metrics(ylt_table, probs):
    """Per layer: mean, PML_p (k-th largest), TVaR_p (mean of the k largest),
    by a full sort. Returns (mean [L], pml [L][n_p], tvar [L][n_p])."""
    lib = _load()
    y = np.ascontiguousarray(ylt_table, dtype=np.float64)
    if y.ndim == 1:
        y = y[None, :]
    L, N = y.shape
    pr = np.ascontiguousarray(probs, dtype=np.float64).reshape(-1)
    mean = np.zeros(L)
    pml = np.zeros((L, pr.size))
    tvar = np.zeros((L, pr.size))
    rc = lib.ara_oracle_metrics(_ptr(y), N, L, _ptr(pr), pr.size, _ptr(mean), _ptr(pml), _ptr(tvar))
    if rc:
        raise OracleError(f"ara_oracle_metrics rejected its inputs (status {rc})")
    return mean, pml, tvar


def tail_count(p: float, n: int) -> int:
    """k = ceil((1-p) N), at least 1 and at most N, with an integer guard."""
    return int(_load().ara_oracle_tail_count(float(p), int(n)))


def num_threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS or all cores)."""
    return int(_load().ara_oracle_num_threads())

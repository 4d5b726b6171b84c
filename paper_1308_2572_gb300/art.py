"""Thin ctypes binding of libart (include/art.h), same names as the C ABI.

Argument marshalling only: every step of aggregate risk analysis runs in the
library's CUDA kernels. Device arguments are CUDA torch tensors (their data
pointers are passed), host arguments numpy arrays or CPU tensors; streams
default to torch's current CUDA stream. There is no fallback: if libart.so
is missing this module raises on first use.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libart.so")

ART_OK, ART_EINVAL, ART_ENOMEM, ART_ECUDA, ART_EID_RANGE, ART_ETIMEOUT, ART_EUNSUPPORTED = range(7)
ART_VARIANT_AUTO, ART_VARIANT_PLAIN, ART_VARIANT_BATCHED, ART_VARIANT_FP64, ART_VARIANT_SKIP, ART_VARIANT_SPARSE = range(6)
ART_LAYOUT_LAYER, ART_LAYOUT_POOL, ART_LAYOUT_POOL64, ART_LAYOUT_GROUP, ART_LAYOUT_SPARSE, ART_LAYOUT_OCC64 = 1, 2, 4, 8, 16, 32
ART_FLAG_L2_PERSIST, ART_FLAG_GRAPH, ART_FLAG_EARLY_EXIT, ART_FLAG_HOST_STAGED = 1, 2, 4, 8

# Every entry point declared in include/art.h.
EXPORTS = ("art_create_portfolio", "art_update_terms", "art_get_terms", "art_set_variant", "art_run_ylt",
           "art_run_ylt_host", "art_metrics", "art_metrics_backward", "art_run_ylt_backward",
           "art_get_device_status", "art_get_footprint", "art_destroy_portfolio", "art_status_string",
           "art_last_cuda_error", "art_version", "art_metrics_noalloc", "art_probe", "art_autotune",
           "art_run_payouts", "art_set_flags", "art_run_ylt_host_metrics", "art_topk", "art_merge_topk")


class LayerTerms(ctypes.Structure):
    _fields_ = [("occ_ret", ctypes.c_double), ("occ_lim", ctypes.c_double),
                ("agg_ret", ctypes.c_double), ("agg_lim", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("layouts", ctypes.c_int32), ("variant", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("trial_tile", ctypes.c_int32), ("cta_threads", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class TuneResult(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("slots", ctypes.c_int32), ("trial_tile", ctypes.c_int32),
                ("cta_threads", ctypes.c_int32), ("sample_ms", ctypes.c_float), ("candidates", ctypes.c_int32),
                ("from_cache", ctypes.c_int32), ("mapping", ctypes.c_int32)]


class ArtError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().art_status_string(status).decode()
        if status == ART_ECUDA or status == ART_ENOMEM:
            msg += f" ({lib().art_last_cuda_error().decode()})"
        super().__init__(f"{where}: {msg}")


_lib = None


def lib():
    """Load libart.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libart.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    st = ctypes.c_int
    sig = {
        "art_create_portfolio": ([i32, i32, P, P, P, P, i32, P, P, P, P, P, P], st),
        "art_update_terms": ([P, P, P, P, P], st),
        "art_get_terms": ([P, P, P, P, P], st),
        "art_set_variant": ([P, i32, i32, i32], st),
        "art_set_flags": ([P, i32], st),
        "art_run_ylt": ([P, i64, P, P, i32, P, P, P], st),
        "art_run_ylt_host": ([P, i64, P, P, i32, P, P], st),
        "art_run_ylt_host_metrics": ([P, i64, P, P, i32, P, P, i32, P, P, P, P], st),
        "art_metrics": ([P, i64, i32, P, i32, P, P, P, P], st),
        "art_metrics_backward": ([P, i64, i32, P, i32, P, P, P, P, P], st),
        "art_metrics_noalloc": ([P, i64, i32, P, i32, P, P, P, P], st),
        "art_topk": ([P, i64, i32, i64, P, P, P], st),
        "art_merge_topk": ([P, P, i32, i32, i64, i64, P, i32, P, P, P], st),
        "art_run_ylt_backward": ([P, i64, P, P, i32, P, P, P, P, P], st),
        "art_get_device_status": ([P, P], st),
        "art_get_footprint": ([P, P, P, P, P, P], st),
        "art_destroy_portfolio": ([P], None),
        "art_status_string": ([st], ctypes.c_char_p),
        "art_last_cuda_error": ([], ctypes.c_char_p),
        "art_version": ([], i32),
        "art_probe": ([i32, i64, i32, P], st),
        "art_autotune": ([P, i64, P, P, i32, P, i32, P, P], st),
        "art_run_payouts": ([P, i32, i64, P, P, i32, P, P, P, P], st),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _check(status: int, where: str) -> None:
    if status != ART_OK:
        raise ArtError(status, where)


def _dptr(t) -> Optional[int]:
    """Device pointer of a CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _hptr(a) -> Optional[int]:
    """Host pointer of a numpy array or CPU tensor (None passes NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if a.is_cuda or not a.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a C-contiguous array")
    return a.ctypes.data


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream or None
    return int(stream) or None


class Portfolio:
    """Owner of an art_portfolio handle; destroyed with the object."""

    def __init__(self, handle: int, n_elt: int, n_layers: int, catalogue_size: int):
        self.handle = handle
        self.n_elt = n_elt
        self.n_layers = n_layers
        self.catalogue_size = catalogue_size

    def close(self) -> None:
        if self.handle:
            art_destroy_portfolio(self)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _h(p) -> int:
    return p.handle if isinstance(p, Portfolio) else p


def art_create_portfolio(catalogue_size: int, elt_losses, elt_mult, elt_ded, elt_lim, layer_elt_off,
                         layer_elt_ids, terms, layouts: int = 0, variant: int = 0, flags: int = 0,
                         trial_tile: int = 0, cta_threads: int = 0, stream=None) -> Portfolio:
    """elt_losses: CUDA float32 [n_elt][C]; elt_mult/ded/lim: host [n_elt]
    (mult may be None); layer_elt_off/ids: host int32; terms: host [L][4]
    (OccR, OccL, AggR, AggL)."""
    n_elt = int(elt_losses.shape[0])
    f32 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
    m, d, l = f32(elt_mult), f32(elt_ded), f32(elt_lim)
    off = np.ascontiguousarray(layer_elt_off, dtype=np.int32)
    ids = np.ascontiguousarray(layer_elt_ids, dtype=np.int32)
    L = off.shape[0] - 1
    tt = np.ascontiguousarray(terms, dtype=np.float64).reshape(L, 4)
    tarr = (LayerTerms * L)(*[LayerTerms(*row) for row in tt])
    opt = Options(layouts, variant, flags, trial_tile, cta_threads)
    out = ctypes.c_void_p()
    rc = lib().art_create_portfolio(int(catalogue_size), n_elt, _dptr(elt_losses), _hptr(m), _hptr(d), _hptr(l), L,
                                    _hptr(off), _hptr(ids), ctypes.cast(tarr, ctypes.c_void_p), ctypes.byref(opt),
                                    _stream(stream), ctypes.byref(out))
    _check(rc, "art_create_portfolio")
    return Portfolio(out.value, n_elt, L, int(catalogue_size))


def art_update_terms(p, elt_mult=None, elt_ded=None, elt_lim=None, terms=None) -> None:
    f32 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
    m, d, l = f32(elt_mult), f32(elt_ded), f32(elt_lim)
    tarr = None
    if terms is not None:
        tt = np.ascontiguousarray(terms, dtype=np.float64).reshape(-1, 4)
        tarr = (LayerTerms * tt.shape[0])(*[LayerTerms(*row) for row in tt])
    rc = lib().art_update_terms(_h(p), _hptr(m), _hptr(d), _hptr(l),
                                None if tarr is None else ctypes.cast(tarr, ctypes.c_void_p))
    _check(rc, "art_update_terms")


def art_get_terms(p):
    """Returns (mult, ded, lim [n_elt] float32, terms [L][4] float64) as applied."""
    m = np.zeros(p.n_elt, np.float32)
    d = np.zeros(p.n_elt, np.float32)
    l = np.zeros(p.n_elt, np.float32)
    tarr = (LayerTerms * p.n_layers)()
    _check(lib().art_get_terms(_h(p), _hptr(m), _hptr(d), _hptr(l), ctypes.cast(tarr, ctypes.c_void_p)),
           "art_get_terms")
    t = np.array([[x.occ_ret, x.occ_lim, x.agg_ret, x.agg_lim] for x in tarr])
    return m, d, l, t


def art_set_variant(p, variant: int, trial_tile: int = 0, cta_threads: int = 0) -> None:
    _check(lib().art_set_variant(_h(p), variant, trial_tile, cta_threads), "art_set_variant")


def art_set_flags(p, flags: int) -> None:
    _check(lib().art_set_flags(_h(p), int(flags)), "art_set_flags")


def art_run_ylt(p, n_trials: int, event_ids, trial_off, events_per_trial: int, ylt, branch=None,
                stream=None) -> None:
    """event_ids: CUDA int32; trial_off: CUDA int64 [T+1] or None (dense, K =
    events_per_trial); ylt: CUDA float64 [L][T]; branch: CUDA uint8 [L][T] or None."""
    rc = lib().art_run_ylt(_h(p), int(n_trials), _dptr(event_ids), _dptr(trial_off), int(events_per_trial),
                           _dptr(ylt), _dptr(branch), _stream(stream))
    _check(rc, "art_run_ylt")


def art_run_ylt_host(p, n_trials: int, event_ids, trial_off, events_per_trial: int, ylt, stream=None) -> None:
    """Host buffers in and out (numpy or CPU tensors; pinned for full speed)."""
    rc = lib().art_run_ylt_host(_h(p), int(n_trials), _hptr(event_ids), _hptr(trial_off), int(events_per_trial),
                                _hptr(ylt), _stream(stream))
    _check(rc, "art_run_ylt_host")


def art_run_ylt_host_metrics(p, n_trials: int, event_ids, trial_off, events_per_trial: int, probs,
                             ylt=None, mean=None, pml=None, tvar=None, stream=None) -> None:
    """Host buffers in (the YET) and out (the YLT if given, mean [L], PML and
    TVaR [L][n_p]; numpy or CPU tensors, pinned for full speed): the YLT stays
    on the device for the metrics."""
    pr = np.ascontiguousarray(probs, dtype=np.float64)
    rc = lib().art_run_ylt_host_metrics(_h(p), int(n_trials), _hptr(event_ids), _hptr(trial_off),
                                        int(events_per_trial), _hptr(ylt), _hptr(pr), pr.size, _hptr(mean),
                                        _hptr(pml), _hptr(tvar), _stream(stream))
    _check(rc, "art_run_ylt_host_metrics")


def art_run_payouts(p, layer: int, n_trials: int, event_ids, trial_off, events_per_trial: int, payouts=None,
                    exhaust=None, ylt=None, stream=None) -> None:
    """Per-event payouts of Algorithm 1's running form for one layer (CUDA
    float64, laid out like event_ids), the position of the event exhausting
    the aggregate limit per trial (CUDA int32 [T], -1 if none) and the trial
    losses (CUDA float64 [T]); any output may be None."""
    rc = lib().art_run_payouts(_h(p), int(layer), int(n_trials), _dptr(event_ids), _dptr(trial_off),
                               int(events_per_trial), _dptr(payouts), _dptr(exhaust), _dptr(ylt), _stream(stream))
    _check(rc, "art_run_payouts")


def art_metrics(ylt, n_trials: int, n_layers: int, probs: Sequence[float], mean=None, pml=None, tvar=None,
                stream=None) -> None:
    pr = np.ascontiguousarray(probs, dtype=np.float64)
    rc = lib().art_metrics(_dptr(ylt), int(n_trials), int(n_layers), _hptr(pr), pr.size, _dptr(mean), _dptr(pml),
                           _dptr(tvar), _stream(stream))
    _check(rc, "art_metrics")


def art_metrics_noalloc(ylt, n_trials: int, n_layers: int, probs: Sequence[float], mean=None, pml=None, tvar=None,
                        stream=None) -> None:
    """art_metrics for callers that cannot allocate device memory: the
    library's fixed 8 MiB static scratch instead of the stream-ordered
    allocator. Calls that overlap on the GPU race on that scratch."""
    pr = np.ascontiguousarray(probs, dtype=np.float64)
    rc = lib().art_metrics_noalloc(_dptr(ylt), int(n_trials), int(n_layers), _hptr(pr), pr.size, _dptr(mean),
                                   _dptr(pml), _dptr(tvar), _stream(stream))
    if rc == ART_EINVAL:
        raise ArtError(rc, "art_metrics_noalloc (invalid arguments, or the layers x probabilities need more than "
                           "the 8 MiB static scratch)")
    _check(rc, "art_metrics_noalloc")


def art_topk(ylt, n_trials: int, n_layers: int, k: int, top, sums=None, stream=None) -> None:
    """One shard's per-layer top-k list (CUDA float64 [L][k]) and loss sums
    (CUDA float64 [L] or None) for a sharded metrics merge."""
    rc = lib().art_topk(_dptr(ylt), int(n_trials), int(n_layers), int(k), _dptr(top), _dptr(sums), _stream(stream))
    _check(rc, "art_topk")


def art_merge_topk(top, sums, n_shards: int, n_layers: int, k: int, n_trials_total: int, probs, mean=None,
                   pml=None, tvar=None) -> None:
    """Host merge of the shards' lists ([S][L][k]) and sums ([S][L]) into the
    whole YLT's mean [L], PML and TVaR [L][n_p] (host arrays or CPU tensors)."""
    pr = np.ascontiguousarray(probs, dtype=np.float64)
    rc = lib().art_merge_topk(_hptr(top), _hptr(sums), int(n_shards), int(n_layers), int(k), int(n_trials_total),
                              _hptr(pr), pr.size, _hptr(mean), _hptr(pml), _hptr(tvar))
    _check(rc, "art_merge_topk")


def art_metrics_backward(ylt, n_trials: int, n_layers: int, probs, pml, grad_mean, grad_tvar, grad_ylt,
                         stream=None) -> None:
    pr = None if probs is None else np.ascontiguousarray(probs, dtype=np.float64)
    rc = lib().art_metrics_backward(_dptr(ylt), int(n_trials), int(n_layers), _hptr(pr), 0 if pr is None else pr.size,
                                    _dptr(pml), _dptr(grad_mean), _dptr(grad_tvar), _dptr(grad_ylt), _stream(stream))
    _check(rc, "art_metrics_backward")


def art_run_ylt_backward(p, n_trials: int, event_ids, trial_off, events_per_trial: int, branch, grad_ylt,
                         grad_terms, grad_mult, stream=None) -> None:
    rc = lib().art_run_ylt_backward(_h(p), int(n_trials), _dptr(event_ids), _dptr(trial_off), int(events_per_trial),
                                    _dptr(branch), _dptr(grad_ylt), _dptr(grad_terms), _dptr(grad_mult),
                                    _stream(stream))
    _check(rc, "art_run_ylt_backward")


def art_autotune(p, n_trials: int, event_ids, trial_off, events_per_trial: int, ylt, sample_trials: int = 0,
                 stream=None) -> dict:
    """Time the variants and tile shapes on a sample of the YET and keep the
    fastest in the portfolio; returns the chosen shape."""
    r = TuneResult()
    rc = lib().art_autotune(_h(p), int(n_trials), _dptr(event_ids), _dptr(trial_off), int(events_per_trial),
                            _dptr(ylt), int(sample_trials), _stream(stream), ctypes.byref(r))
    _check(rc, "art_autotune")
    return {f: getattr(r, f) for f, _ in TuneResult._fields_}


def art_get_device_status(p, stream=None) -> int:
    """Synchronises the stream; returns ART_OK, ART_EID_RANGE or ART_EINVAL."""
    return int(lib().art_get_device_status(_h(p), _stream(stream)))


def art_get_footprint(p):
    """Returns (layer, pool, pool64, group, sparse) bytes held on the device."""
    v = [ctypes.c_int64() for _ in range(5)]
    _check(lib().art_get_footprint(_h(p), *[ctypes.byref(x) for x in v]), "art_get_footprint")
    return tuple(x.value for x in v)


def art_destroy_portfolio(p) -> None:
    lib().art_destroy_portfolio(_h(p))


def art_status_string(status: int) -> str:
    return lib().art_status_string(int(status)).decode()


ART_PROBE_STREAM, ART_PROBE_GATHER32, ART_PROBE_GATHER64, ART_PROBE_GATHER4, ART_PROBE_FP64ADD = range(5)


def art_probe(kind: int, nbytes: int = 64 << 20, reps: int = 5) -> float:
    """Measured rate (GB/s, or GFLOP/s for the FP64 probe); see include/art.h."""
    out = ctypes.c_double()
    _check(lib().art_probe(int(kind), int(nbytes), int(reps), ctypes.byref(out)), "art_probe")
    return out.value


def art_version() -> int:
    return int(lib().art_version())


# ---------------------------------------------------------------- helpers

def portfolio_from_workload(w, device="cuda", **kw) -> Portfolio:
    """Build a portfolio from a workloads.Workload (the tables go to the
    device once, then the library re-lays them out)."""
    import torch
    port = w.portfolio
    tab = torch.from_numpy(port.elt_losses).to(device)
    terms = np.stack([port.occ_ret, port.occ_lim, port.agg_ret, port.agg_lim], axis=1)
    p = art_create_portfolio(port.catalogue_size, tab, port.elt_mult, port.elt_ded, port.elt_lim,
                             port.layer_elt_off, port.layer_elt_ids, terms, **kw)
    del tab
    return p

"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws inputs only: it holds none of the method's arithmetic and
is the one piece of code that both the CUDA path's callers and the FP64
oracle's callers share. The paper's YETs and ELTs are proprietary; these
stand in for them with the shapes of Section III (catalogue of 2,000,000
events, 1,000,000 trials of about 1,000 events, layers of 1-32 ELTs of
10,000-50,000 non-zero losses).

Recipes (seed = 13082572 + config number; numpy PCG64 streams spawned per
part so that a smaller trial count draws a prefix of the same YET):

  c0   catalogue 100,000; 10,000 trials x 1,000 events; 1 layer of 3 ELTs,
       each 10,000 distinct non-zero ids with lognormal(12, 2) losses;
       D_e / Lim_e = 5th / 99th percentile of the ELT's non-zero losses;
       OccR 1e5, OccL 5e6, AggR 1e6, AggL 2e7.
  c0u  c0 with AggR 1.5e8, AggL 1e8 (aggregate terms straddle the median
       aggregate, so the layer is not capped on every trial).
  c1   catalogue 2,000,000; 1,000,000 trials x 1,000 events; 1 layer of 16
       ELTs with 20,000 non-zero lognormal(12, 2) losses; c0's term rules.
  c1u  c1 with AggR 9e7, AggL 5e7.
  c2   catalogue 2,000,000; 1,000,000 trials of clamp(Poisson(1000), 200,
       2000) events (CSR); pool of 256 ELTs with U{10,000..50,000} non-zero
       lognormal(12, 2.5) losses; 64 layers of U{1..32} distinct pool ELTs;
       OccR ~ logU[1e5, 1e6], OccL = OccR logU[10, 100], AggR ~ logU[2e7,
       3e8], AggL = AggR logU[1.5, 10].
  c3   c1's YET and 16 ELTs, multipliers 1; 8 layers, layer j covering ELTs
       (2j + i) mod 16 for i = 0..7; OccR 1e5, OccL 5e6, AggR 3e7 + 5e6 j,
       AggL 3e7.
  c4   catalogue 2,000,000; 1,000,000 trials x 1,000 events; pool of 512 ELTs
       with U{10,000..50,000} non-zero lognormal(13, 2.5) losses; 128 layers
       of U{4..32} ELTs; c2's term ranges with the aggregate ranges x 3.

Event ids are uniform over the catalogue, with replacement. Timestamps are
drawn only on request (uniform [0, 365), sorted within each trial); the
year loss does not depend on them.

Occurrence terms and ELT terms are returned already rounded to FP32 (the
precision the kernels apply them in); aggregate terms stay FP64.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

SEED_BASE = 13082572


@dataclasses.dataclass
class Portfolio:
    catalogue_size: int
    elt_losses: np.ndarray          # [n_elt][catalogue_size] float32, direct-access tables
    elt_mult: np.ndarray            # [n_elt] float32
    elt_ded: np.ndarray             # [n_elt] float32
    elt_lim: np.ndarray             # [n_elt] float32 (may be +inf)
    layer_elt_off: np.ndarray       # [n_layers + 1] int32
    layer_elt_ids: np.ndarray       # int32
    occ_ret: np.ndarray             # [n_layers] float64 (FP32-representable)
    occ_lim: np.ndarray             # [n_layers] float64 (FP32-representable or +inf)
    agg_ret: np.ndarray             # [n_layers] float64
    agg_lim: np.ndarray             # [n_layers] float64 (may be +inf)

    @property
    def n_elt(self) -> int:
        return int(self.elt_losses.shape[0])

    @property
    def n_layers(self) -> int:
        return int(self.layer_elt_off.shape[0] - 1)

    def elts_per_layer(self) -> np.ndarray:
        return np.diff(self.layer_elt_off.astype(np.int64))


@dataclasses.dataclass
class YET:
    n_trials: int
    event_ids: np.ndarray                   # int32, [n_trials * K] (dense) or [total] (CSR)
    events_per_trial: int = 0               # K for a dense YET, 0 for CSR
    trial_off: Optional[np.ndarray] = None  # [n_trials + 1] int64 for CSR, None for dense
    timestamps: Optional[np.ndarray] = None

    @property
    def n_events(self) -> int:
        return int(self.event_ids.shape[0])

    def offsets(self) -> np.ndarray:
        """Trial offsets as int64 [n_trials + 1], for dense YETs too."""
        if self.trial_off is not None:
            return self.trial_off
        return np.arange(self.n_trials + 1, dtype=np.int64) * self.events_per_trial

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets())


@dataclasses.dataclass
class Workload:
    name: str
    portfolio: Portfolio
    yet: YET
    probs: np.ndarray

    def oracle_problem(self) -> dict:
        """Arguments in the form the oracle's wrappers take."""
        p, y = self.portfolio, self.yet
        d = dict(catalogue_size=p.catalogue_size, elt_losses=p.elt_losses,
                 elt_mult=p.elt_mult.astype(np.float64), elt_ded=p.elt_ded.astype(np.float64),
                 elt_lim=p.elt_lim.astype(np.float64), layer_elt_off=p.layer_elt_off,
                 layer_elt_ids=p.layer_elt_ids, occ_ret=p.occ_ret, occ_lim=p.occ_lim,
                 agg_ret=p.agg_ret, agg_lim=p.agg_lim, event_ids=y.event_ids)
        if y.trial_off is not None:
            d["trial_off"] = y.trial_off
        else:
            d["events_per_trial"] = y.events_per_trial
            d["n_trials"] = y.n_trials
        return d

    def lookups(self) -> int:
        """Trial-event x ELT lookups of one pass: sum_t K_t * sum_j |E_j|."""
        return int(self.yet.n_events) * int(self.portfolio.layer_elt_ids.shape[0])


def _streams(seed: int, n: int):
    return [np.random.Generator(np.random.PCG64(s)) for s in np.random.SeedSequence(seed).spawn(n)]


def _f32(x) -> np.ndarray:
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def sparse_elts(rng, n_elt: int, catalogue: int, nnz, mu: float, sigma: float):
    """Per ELT: distinct non-zero event ids and FP32 lognormal losses."""
    out = []
    for e in range(n_elt):
        k = int(nnz[e]) if np.ndim(nnz) else int(nnz)
        ids = np.sort(rng.choice(catalogue, size=k, replace=False)).astype(np.int32)
        loss = rng.lognormal(mean=mu, sigma=sigma, size=k).astype(np.float32)
        out.append((ids, loss))
    return out


def dense_tables(sparse, catalogue: int) -> np.ndarray:
    """Direct-access tables [n_elt][catalogue] float32, zero where absent."""
    tab = np.zeros((len(sparse), catalogue), dtype=np.float32)
    for e, (ids, loss) in enumerate(sparse):
        tab[e, ids] = loss
    return tab


def percentile_terms(sparse):
    """D_e, Lim_e = 5th and 99th percentile of the ELT's non-zero losses
    (numpy linear percentile in FP64), rounded to FP32."""
    ded = np.array([np.percentile(l.astype(np.float64), 5) for _, l in sparse], dtype=np.float32)
    lim = np.array([np.percentile(l.astype(np.float64), 99) for _, l in sparse], dtype=np.float32)
    return ded, lim


def dense_yet(rng, n_trials: int, k: int, catalogue: int, chunk: int = 1 << 24) -> np.ndarray:
    ids = np.empty(n_trials * k, dtype=np.int32)
    for s in range(0, ids.size, chunk):
        e = min(ids.size, s + chunk)
        ids[s:e] = rng.integers(0, catalogue, size=e - s, dtype=np.int32)
    return ids


def sorted_timestamps(rng, lengths: np.ndarray) -> np.ndarray:
    ts = rng.uniform(0.0, 365.0, size=int(lengths.sum())).astype(np.float32)
    off = np.concatenate([[0], np.cumsum(lengths)])
    for t in range(lengths.size):
        ts[off[t]:off[t + 1]].sort()
    return ts


def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=size))


def _portfolio(catalogue, tables, mult, ded, lim, layer_lists, occ_ret, occ_lim, agg_ret, agg_lim):
    off = np.zeros(len(layer_lists) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(l) for l in layer_lists])
    ids = np.concatenate([np.asarray(l, dtype=np.int32) for l in layer_lists]) if layer_lists else np.zeros(0, np.int32)
    return Portfolio(catalogue_size=catalogue, elt_losses=tables,
                     elt_mult=np.asarray(mult, dtype=np.float32), elt_ded=np.asarray(ded, dtype=np.float32),
                     elt_lim=np.asarray(lim, dtype=np.float32), layer_elt_off=off, layer_elt_ids=ids,
                     occ_ret=_f32(occ_ret), occ_lim=_f32(occ_lim),
                     agg_ret=np.asarray(agg_ret, dtype=np.float64), agg_lim=np.asarray(agg_lim, dtype=np.float64))


def make(name: str, n_trials: Optional[int] = None, with_timestamps: bool = False, shard: int = 0) -> Workload:
    """Build a named workload (c0, c0u, c1, c1u, c2, c3, c4); n_trials, when
    given, keeps the first n_trials trials of the full YET. shard s > 0 draws
    the YET (and its timestamps) from stream 3 + s instead: the same
    portfolio with another YET of the same recipe, one per GPU of a run that
    splits its trials between GPUs (shard 0 is the workload itself)."""
    base = name.rstrip("u")
    cfg = int(base[1:])
    seed = SEED_BASE + cfg
    streams = _streams(seed, 4 + max(0, int(shard)))
    r_elt, r_layer, r_yet, r_ts = streams[:4]
    if shard > 0:
        r_yet = r_ts = streams[3 + shard]
    probs = np.array([0.99])

    if base in ("c0", "c1", "c3"):
        C, T, K = (100_000, 10_000, 1000) if base == "c0" else (2_000_000, 1_000_000, 1000)
        n_elt, nnz = (3, 10_000) if base == "c0" else (16, 20_000)
        sp = sparse_elts(r_elt, n_elt, C, nnz, 12.0, 2.0)
        tables = dense_tables(sp, C)
        ded, lim = percentile_terms(sp)
        mult = np.ones(n_elt, dtype=np.float32)
        if base == "c3":
            lists = [[(2 * j + i) % 16 for i in range(8)] for j in range(8)]
            occ_ret, occ_lim = np.full(8, 1e5), np.full(8, 5e6)
            agg_ret = 3e7 + 5e6 * np.arange(8)
            agg_lim = np.full(8, 3e7)
        else:
            lists = [list(range(n_elt))]
            occ_ret, occ_lim = [1e5], [5e6]
            if name == "c0u":
                agg_ret, agg_lim = [1.5e8], [1e8]
            elif name == "c1u":
                agg_ret, agg_lim = [9e7], [5e7]
            else:
                agg_ret, agg_lim = [1e6], [2e7]
        port = _portfolio(C, tables, mult, ded, lim, lists, occ_ret, occ_lim, agg_ret, agg_lim)
        T = T if n_trials is None else int(n_trials)
        yet = YET(n_trials=T, event_ids=dense_yet(r_yet, T, K, C), events_per_trial=K)
    elif base in ("c2", "c4"):
        C = 2_000_000
        n_pool, mu, n_layers, lo_n = (256, 12.0, 64, 1) if base == "c2" else (512, 13.0, 128, 4)
        agg_scale = 1.0 if base == "c2" else 3.0
        nnz = r_elt.integers(10_000, 50_001, size=n_pool)
        sp = sparse_elts(r_elt, n_pool, C, nnz, mu, 2.5)
        tables = dense_tables(sp, C)
        ded, lim = percentile_terms(sp)
        mult = np.ones(n_pool, dtype=np.float32)
        sizes = r_layer.integers(lo_n, 33, size=n_layers)
        lists = [np.sort(r_layer.choice(n_pool, size=int(s), replace=False)) for s in sizes]
        occ_ret = _log_uniform(r_layer, 1e5, 1e6, n_layers)
        occ_lim = occ_ret * _log_uniform(r_layer, 10.0, 100.0, n_layers)
        agg_ret = _log_uniform(r_layer, 2e7 * agg_scale, 3e8 * agg_scale, n_layers)
        agg_lim = agg_ret * _log_uniform(r_layer, 1.5, 10.0, n_layers)
        port = _portfolio(C, tables, mult, ded, lim, lists, occ_ret, occ_lim, agg_ret, agg_lim)
        T = 1_000_000 if n_trials is None else int(n_trials)
        if base == "c2":
            lengths = np.clip(r_yet.poisson(1000, size=T), 200, 2000).astype(np.int64)
            off = np.zeros(T + 1, dtype=np.int64)
            off[1:] = np.cumsum(lengths)
            ids = dense_yet(r_yet, 1, int(off[-1]), C)
            yet = YET(n_trials=T, event_ids=ids, trial_off=off)
        else:
            yet = YET(n_trials=T, event_ids=dense_yet(r_yet, T, 1000, C), events_per_trial=1000)
            probs = np.array([0.99, 0.996, 0.999])
    else:
        raise ValueError(f"unknown workload {name!r}")
    if with_timestamps:
        yet.timestamps = sorted_timestamps(r_ts, yet.lengths())
    return Workload(name=name, portfolio=port, yet=yet, probs=probs)


def random_case(seed: int, catalogue: int = 97, n_elt: int = 5, n_layers: int = 3,
                n_trials: int = 37, min_len: int = 0, max_len: int = 70, nnz_frac: float = 0.3,
                max_elts_per_layer: Optional[int] = None, inf_limits: bool = False,
                dense_k: Optional[int] = None, mult_range=(1.0, 1.0)) -> Workload:
    """A small random workload with ragged trials (empty ones included when
    min_len is 0), uneven layers and terms scaled to the losses, for parity
    tests that must span several tiles and a ragged tail."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nnz = max(1, int(nnz_frac * catalogue))
    sp = sparse_elts(rng, n_elt, catalogue, np.full(n_elt, nnz), 10.0, 1.5)
    tables = dense_tables(sp, catalogue)
    ded, lim = percentile_terms(sp)
    mult = rng.uniform(mult_range[0], mult_range[1], size=n_elt).astype(np.float32)
    hi = n_elt if max_elts_per_layer is None else min(n_elt, max_elts_per_layer)
    lists = [np.sort(rng.choice(n_elt, size=int(rng.integers(1, hi + 1)), replace=False)) for _ in range(n_layers)]
    typical = float(np.median(np.concatenate([l for _, l in sp])))
    occ_ret = typical * rng.uniform(0.2, 2.0, n_layers)
    occ_lim = occ_ret * rng.uniform(2.0, 20.0, n_layers)
    mean_len = 0.5 * (min_len + max_len) if dense_k is None else dense_k
    scale = typical * max(1.0, mean_len) * nnz_frac * 0.5
    agg_ret = scale * rng.uniform(0.05, 0.5, n_layers)
    agg_lim = scale * rng.uniform(0.2, 1.0, n_layers)
    if inf_limits:
        lim[::2] = np.inf
        occ_lim[::2] = np.inf
        agg_lim[1::2] = np.inf
    port = _portfolio(catalogue, tables, mult, ded, lim, lists, occ_ret, occ_lim, agg_ret, agg_lim)
    if dense_k is not None:
        yet = YET(n_trials=n_trials, event_ids=dense_yet(rng, n_trials, dense_k, catalogue), events_per_trial=dense_k)
    else:
        lengths = rng.integers(min_len, max_len + 1, size=n_trials).astype(np.int64)
        off = np.zeros(n_trials + 1, dtype=np.int64)
        off[1:] = np.cumsum(lengths)
        yet = YET(n_trials=n_trials, event_ids=dense_yet(rng, 1, int(off[-1]), catalogue) if off[-1] else np.zeros(0, np.int32), trial_off=off)
    return Workload(name=f"random{seed}", portfolio=port, yet=yet, probs=np.array([0.9, 0.99]))

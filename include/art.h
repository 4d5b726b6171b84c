/*
 * art.h -- C ABI of libart, GB300-native aggregate risk analysis.
 *
 * Method: Bahl, Baltzer, Rau-Chaplin, Varghese, Whiteway, "Achieving Speedup
 * in Aggregate Risk Analysis using Multiple GPUs" (arXiv:1308.2572).
 * A Year Event Table (YET: per trial, a list of event ids), a set of Event
 * Loss Tables (ELTs: event id -> loss, plus per-ELT financial terms) and a
 * set of excess-of-loss layers (each covering some ELTs, with occurrence and
 * aggregate retentions and limits) give a Year Loss Table YLT[layer][trial]
 * (Section II, Algorithm 1). From the YLT come the expected loss, PML and
 * TVaR (Section I).
 *
 * Conventions shared by every entry point:
 *  - Pointers named *_dev are device pointers on the current CUDA device;
 *    pointers named *_host are host pointers. Caller buffers stay owned by
 *    the caller; the library never frees them and keeps no reference to them
 *    after the call returns, except where a call says so.
 *  - Calls that take a stream are stream-ordered and asynchronous: they
 *    enqueue work and return. A NULL stream is the legacy default stream.
 *  - Host-side validation errors return at once (ART_EINVAL) and enqueue
 *    nothing. Errors found on the device (an event id outside the catalogue)
 *    never trap: the offending event counts as zero loss, a device flag is
 *    set, and art_get_device_status reports ART_EID_RANGE.
 *  - Every piecewise-linear term is XL(v; R, L) = min(max(v - R, 0), L);
 *    limits may be +INFINITY (an unlimited cover).
 *  - No entry point waits on other CTAs or other GPUs; there are no spin
 *    waits in any kernel of this library.
 *  - A portfolio belongs to the device that was current when it was created;
 *    call the entry points that take it with that device current. A
 *    portfolio is not thread-safe (its graph cache, staging buffers and work
 *    counter are shared): use it from one host thread at a time, and order
 *    run calls that share it on one stream (they share the work counter).
 *  - Results are deterministic: the same inputs, variant and tile shape give
 *    bitwise-equal outputs (no atomics take part in any sum).
 */
#ifndef ART_H
#define ART_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#if defined(__GNUC__)
#define ART_API __attribute__((visibility("default")))
#else
#define ART_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ART_OK = 0,
    ART_EINVAL = 1,        /* an argument failed host-side validation        */
    ART_ENOMEM = 2,        /* a device allocation failed                      */
    ART_ECUDA = 3,         /* a CUDA runtime call failed                      */
    ART_EID_RANGE = 4,     /* the device saw an event id outside [0, C)       */
    ART_ETIMEOUT = 5,      /* reserved: a bounded wait gave up                */
    ART_EUNSUPPORTED = 6   /* the portfolio lacks the layout this call needs  */
} art_status;

/* Opaque portfolio: the library's own device copies of the ELTs in the
 * layouts its kernels read, plus the FP32-rounded terms. */
typedef struct art_portfolio art_portfolio;

/* Layer terms T = (OccR, OccL, AggR, AggL) of Section II. Retentions must be
 * finite and >= 0; limits > 0 or +INFINITY. OccR and OccL are rounded to
 * FP32 (the precision the occurrence test runs in); AggR and AggL stay FP64. */
typedef struct {
    double occ_ret;
    double occ_lim;
    double agg_ret;
    double agg_lim;
} art_layer_terms;

/* Kernel variants for art_run_ylt. */
enum {
    ART_VARIANT_AUTO = 0,     /* batched when the pool layout exists, else plain          */
    ART_VARIANT_PLAIN = 1,    /* one launch per layer over a per-layer event-major table  */
    ART_VARIANT_BATCHED = 2,  /* one persistent launch over all layers (pool table)       */
    ART_VARIANT_FP64 = 3,     /* all-FP64 arithmetic: per call, FP64 occurrence losses of
                                 every catalogue event, then one trial pass per run of
                                 <= 4 layers that sums them exactly (integer fixed point,
                                 one FP64 rounding per trial) and applies the aggregate
                                 terms in FP64 (ART_LAYOUT_OCC64); else batched over the
                                 FP64 pool with FP64 sums (ART_LAYOUT_POOL64)             */
    ART_VARIANT_SKIP = 4,     /* per call, the occurrence loss of every catalogue event
                                 for every layer (one build launch, from the CSR of the
                                 non-zero losses when ART_LAYOUT_SPARSE is present, else
                                 from the per-layer tables; the same values bit for bit),
                                 then one trial pass per run of <= 8 layers that skips
                                 events with zero occurrence loss (bitmap)               */
    ART_VARIANT_SPARSE = 5    /* one persistent launch over all layers, reading an
                                 event-major CSR of the non-zero losses (compressed ELTs) */
};

/* Layouts built by art_create_portfolio (bit mask). */
enum {
    ART_LAYOUT_LAYER = 1,     /* per layer: [C][n_pad] FP32, the layer's ELTs side by side;
                                 plus, per run of <= 8 layers, a [C + 1][<= 8] FP32
                                 occurrence-loss table and bitmap written by the skip
                                 variant on every call (counted with the layer bytes)     */
    ART_LAYOUT_POOL = 2,      /* all ELTs:  [C][n_elt_pad] FP32, shared by every layer     */
    ART_LAYOUT_POOL64 = 4,    /* all ELTs:  [C][n_elt_pad] FP64 (precision study)          */
    ART_LAYOUT_GROUP = 8,     /* per layer group (<= 8 layers, <= 32 ELTs together):
                                 [C][n_pad] FP32 over the group's ELTs plus a C-bit
                                 occupancy bitmap; read by art_run_ylt_backward           */
    ART_LAYOUT_SPARSE = 16,   /* all ELTs: event-major CSR of the non-zero losses
                                 (C + 1 offsets, 8 bytes per non-zero loss); also the
                                 source of the skip and all-FP64 variants' per-call
                                 occurrence tables                                         */
    ART_LAYOUT_OCC64 = 32     /* with ART_LAYOUT_LAYER: FP64 occurrence-loss tables
                                 ([C + 1][<= 4] 8-byte entries per run of <= 4 layers) and
                                 bitmaps, written by the all-FP64 variant on every call
                                 (FP64 values, then packed in place into fixed-point
                                 words); that variant then uses them instead of the
                                 FP64 pool (counted with the pool64 bytes)                 */
};

/* Flags. */
enum {
    ART_FLAG_L2_PERSIST = 1,  /* set a persisting L2 access-policy window over the hot
                                 table on the stream passed to each run call (the skip
                                 variant: over each occurrence group's table during
                                 that group's pass; the window is cleared afterwards) */
    ART_FLAG_GRAPH = 2,       /* art_run_ylt captures its launches (any variant) in a CUDA
                                 graph once per argument set and replays it            */
    ART_FLAG_EARLY_EXIT = 4,  /* skip variant: stop reading a trial once every layer of the
                                 group has reached its aggregate cap (the aggregate never
                                 decreases, so the loss is AggL); same results within FP32
                                 rounding of the cap, far fewer lookups on capped trials  */
    ART_FLAG_HOST_STAGED = 8  /* art_run_ylt_host*: always copy the YET to the device in
                                 staged chunks, never read it in place (see
                                 art_run_ylt_host)                                          */
};

typedef struct {
    int32_t layouts;          /* ART_LAYOUT_* mask; 0 means LAYER | POOL | GROUP | SPARSE      */
    int32_t variant;          /* ART_VARIANT_*                                                */
    int32_t flags;            /* ART_FLAG_*                                                   */
    int32_t trial_tile;       /* batched: trials per work unit (0 = autotune / default)       */
    int32_t cta_threads;      /* batched: threads per CTA (0 = default)                       */
    int32_t reserved[3];
} art_options;

/*
 * art_create_portfolio -- the preprocessing stage (Section II: YET, ELT and
 * layers loaded into memory; Section III: ELTs as direct-access tables).
 *
 *  catalogue_size     C, number of event ids; ids are 0..C-1. 1 <= C < 2^31.
 *  n_elt              number of ELTs, 1..4096.
 *  elt_losses_dev     [n_elt][C] FP32 direct-access tables (row e is ELT e,
 *                     zero where the ELT has no loss); device memory, read
 *                     during this call only. Values must be finite, >= 0.
 *  elt_mult_host,     [n_elt] FP32 financial terms of each ELT: the loss
 *  elt_ded_host,      becomes F_e(y) = XL(m_e y; D_e, Lim_e) (the paper names
 *  elt_lim_host       per-ELT terms but not their form; this is the reading).
 *                     m_e, D_e finite >= 0; Lim_e > 0 or +INFINITY.
 *                     elt_mult_host may be NULL (all 1).
 *  n_layers           1..65536 (art_metrics takes at most 65535 per call).
 *  layer_elt_off_host [n_layers + 1], starts at 0, non-decreasing; layer j
 *                     covers layer_elt_ids_host[off[j] .. off[j+1]), 1..32
 *                     distinct ELT ids per layer.
 *  terms_host         [n_layers] layer terms.
 *  opt                NULL for defaults.
 *  stream             stream the table builds run on; the call returns after
 *                     they complete (the caller's buffer may be reused).
 *  out                receives the portfolio; destroy with art_destroy_portfolio.
 * Errors: ART_EINVAL (validation), ART_ENOMEM, ART_ECUDA.
 */
ART_API art_status art_create_portfolio(int32_t catalogue_size, int32_t n_elt, const float* elt_losses_dev,
                                const float* elt_mult_host, const float* elt_ded_host,
                                const float* elt_lim_host, int32_t n_layers,
                                const int32_t* layer_elt_off_host, const int32_t* layer_elt_ids_host,
                                const art_layer_terms* terms_host, const art_options* opt,
                                cudaStream_t stream, art_portfolio** out);

/* Replace the terms without rebuilding tables (pricing loops, finite
 * differences). The terms are those of Section II: per ELT the financial
 * terms (multiplier, deductible, limit), per layer the occurrence and
 * aggregate retentions and limits. Any pointer may be NULL to keep those
 * terms. Same validation and rounding as art_create_portfolio. Takes effect
 * for calls enqueued afterwards on any stream; the caller orders it against
 * calls in flight. Errors: ART_EINVAL (NULL portfolio or invalid terms;
 * nothing changes), ART_ECUDA (the device copy could not be refreshed;
 * destroy the portfolio). */
ART_API art_status art_update_terms(art_portfolio* p, const float* elt_mult_host, const float* elt_ded_host,
                            const float* elt_lim_host, const art_layer_terms* terms_host);

/* Read back the Section II terms as the kernels apply them (after FP32
 * rounding): elt_* [n_elt], terms_host [n_layers], caller-owned host
 * arrays. Any pointer may be NULL. Errors: ART_EINVAL (NULL portfolio). */
ART_API art_status art_get_terms(const art_portfolio* p, float* elt_mult_host, float* elt_ded_host,
                         float* elt_lim_host, art_layer_terms* terms_host);

/* Replace the portfolio's ART_FLAG_* flags (execution options with no
 * counterpart in the paper; ART_FLAG_L2_PERSIST takes effect only if it was
 * set at creation, which reserves the persisting L2 area). Drops a captured
 * graph. Errors: ART_EINVAL (NULL portfolio or an unknown flag bit). */
ART_API art_status art_set_flags(art_portfolio* p, int32_t flags);

/* Select the kernel variant (ART_VARIANT_*; every variant computes
 * Algorithm 1 of Section II) and the batched tile shape; 0 keeps the
 * current value of a tile parameter. Drops a captured graph. Errors:
 * ART_EINVAL (NULL portfolio, unknown variant, negative tile, CTA size not a
 * multiple of 32 or above 1024), ART_EUNSUPPORTED (the variant's layout was
 * not built). */
ART_API art_status art_set_variant(art_portfolio* p, int32_t variant, int32_t trial_tile, int32_t cta_threads);

/*
 * art_run_ylt -- the simulation stage (Section II, Algorithm 1, steps 1-4):
 * for every layer j and trial t,
 *     x_d = sum_{e in E_j} F_e(l_e[E_{t,d}])   FP32, ELT order
 *     o_d = XL(x_d; OccR_j, OccL_j)            FP32
 *     S   = sum_d o_d                          FP64
 *     Y   = XL(S; AggR_j, AggL_j)              FP64
 * Y equals the trial loss lr of Algorithm 1: its per-event differences of the
 * aggregate terms telescope to XL(S; AggR, AggL) because AggR >= 0, so event
 * order (and the timestamps) does not change Y.
 *
 *  n_trials           0 <= T <= 2^40 (0 is a no-op); a dense YET also needs
 *                     T K <= 2^62, and every trial must hold fewer than 2^31
 *                     events (the kernels index positions within a trial in
 *                     32 bits).
 *  event_ids_dev      int32 event ids. Dense: [T][K]. CSR: trial t is
 *                     event_ids_dev[off[t] .. off[t+1]); must not be NULL for
 *                     CSR input, even when every trial is empty.
 *  trial_off_dev      NULL for a dense YET, else [T+1] int64, off[0] = 0,
 *                     non-decreasing (checked on the device: a decreasing pair
 *                     is treated as an empty trial and flags ART_EINVAL via
 *                     art_get_device_status).
 *  events_per_trial   K for a dense YET (>= 0), ignored for CSR.
 *  ylt_dev            [n_layers][T] FP64 output.
 *  branch_dev         NULL, or [n_layers][T] uint8 output: 0 when S <= AggR,
 *                     1 when AggR < S < AggR + AggL, 2 above (the aggregate
 *                     branch art_run_ylt_backward needs).
 * Errors: ART_EINVAL, ART_EUNSUPPORTED (variant's layout not built), ART_ECUDA.
 */
ART_API art_status art_run_ylt(art_portfolio* p, int64_t n_trials, const int32_t* event_ids_dev,
                       const int64_t* trial_off_dev, int32_t events_per_trial, double* ylt_dev,
                       uint8_t* branch_dev, cudaStream_t stream);

/*
 * art_run_ylt_host -- art_run_ylt from host buffers, two ways. (1) In
 * place: when the YET buffers are page-locked host memory mapped into the
 * current device (cudaHostAlloc, cudaHostRegister with mapping, a pinned
 * buffer under unified addressing: cudaHostGetDevicePointer succeeds) and
 * the variant reads every event id once per call (the skip and all-FP64
 * variants with one occurrence group, the plain variant with one layer),
 * the forward reads the ids from host memory over the host link, into a
 * device YLT the portfolio keeps, which is then copied into ylt_host. (2)
 * Staged, otherwise or with ART_FLAG_HOST_STAGED: the YET is copied to the
 * device in chunks of trials on the given stream, each chunk's YLT rows are
 * computed and copied back into ylt_host ([n_layers][T] FP64). The
 * portfolio owns the device YLT and the staging buffers (grown on demand,
 * freed with the portfolio). Both give the same results. Blocks until the
 * result is in ylt_host. Dense YETs only (trial_off NULL) or CSR with host
 * offsets. Pinned host memory gives full link bandwidth.
 * The chunks stand for the paper's chunked reads of the YET (Section III);
 * the result is that of art_run_ylt (Algorithm 1, Section II). Host offsets
 * are checked on the host (off[0] = 0, non-decreasing) before any copy.
 * Errors: ART_EINVAL, ART_EUNSUPPORTED, ART_ECUDA (including a failed
 * staging allocation).
 */
ART_API art_status art_run_ylt_host(art_portfolio* p, int64_t n_trials, const int32_t* event_ids_host,
                            const int64_t* trial_off_host, int32_t events_per_trial,
                            double* ylt_host, cudaStream_t stream);

/*
 * art_run_ylt_host_metrics -- the simulation stage and the financial
 * functions from host buffers in one call (Section II, Algorithm 1 on a YET
 * read in chunks as in Section III; Section I, PML and TVaR of the YLT): the
 * YET is read in place or staged in chunks as in art_run_ylt_host, the whole
 * YLT is kept on the device, art_metrics runs on it there, and only the
 * results come back. The YLT never makes a device-host-device round trip.
 *  ylt_host      NULL, or [n_layers][T] FP64 host output (the YLT as well).
 *  probs_host    [n_p] probabilities in (0, 1), 1 <= n_p <= 8.
 *  mean_host     [n_layers], pml_host and tvar_host [n_layers][n_p]: FP64
 *                host outputs, each may be NULL.
 * Limits: those of art_run_ylt_host and of art_metrics (1 <= T <= 2^31 - 1,
 * n_layers <= 65535). The portfolio owns a device array for the whole YLT
 * ([n_layers][T] FP64) and the metrics' scratch besides the staging buffers,
 * grown on demand and freed with the portfolio, so that repeated calls of
 * the same size allocate nothing. Blocks until the results are in host
 * memory. Results equal
 * art_run_ylt followed by art_metrics. Errors: ART_EINVAL, ART_EUNSUPPORTED,
 * ART_ECUDA (including a failed allocation).
 */
ART_API art_status art_run_ylt_host_metrics(art_portfolio* p, int64_t n_trials, const int32_t* event_ids_host,
                                            const int64_t* trial_off_host, int32_t events_per_trial,
                                            double* ylt_host, const double* probs_host, int32_t n_p,
                                            double* mean_host, double* pml_host, double* tvar_host,
                                            cudaStream_t stream);

/*
 * art_run_payouts -- Algorithm 1's running form for one layer (Section II:
 * the cumulative sum of the occurrence-net losses, the aggregate terms on
 * every cumulative value, the per-event difference, and the trial loss as
 * their sum). For layer j and every trial, in trial order,
 *     C_d = sum_{i <= d} o_i                        FP64
 *     p_d = XL(C_d; AggR, AggL) - XL(C_{d-1}; AggR, AggL),  C_0 = 0
 * with o_i as in art_run_ylt. Unlike the trial loss, the payouts depend on
 * the order of the events (the aggregate limit runs out part way).
 *  layer          0 .. n_layers-1 (needs the ART_LAYOUT_LAYER tables).
 *  payouts_dev    NULL, or one FP64 per event of the YET, laid out like
 *                 event_ids_dev (dense [T][K] or CSR positions).
 *  exhaust_dev    NULL, or [T] int32: the 0-based position within the trial
 *                 of the first event with C_d - AggR >= AggL (the event that
 *                 exhausts the aggregate limit), -1 if none.
 *  ylt_dev        NULL, or [T] FP64: XL(C_K; AggR, AggL), the sum of the p_d.
 * Runs FP64 arithmetic per event: a reporting path, much slower than
 * art_run_ylt. Errors: ART_EINVAL, ART_EUNSUPPORTED, ART_ECUDA.
 */
ART_API art_status art_run_payouts(art_portfolio* p, int32_t layer, int64_t n_trials, const int32_t* event_ids_dev,
                                   const int64_t* trial_off_dev, int32_t events_per_trial, double* payouts_dev,
                                   int32_t* exhaust_dev, double* ylt_dev, cudaStream_t stream);

/*
 * art_metrics -- financial functions on the YLT (Section I: PML and TVaR;
 * Section II: "financial functions or filters" on the trial losses).
 * Per layer j: mean_j = (1/T) sum_t Y_{j,t}; with k = ceil((1 - p) T)
 * (at least 1; a (1-p)T within 1e-9 T of an integer is taken as that
 * integer), PML_p = the k-th largest Y_{j,.} and TVaR_p = the mean of the k
 * largest. Exact selection (radix select on the FP64 bit patterns), FP64 sums.
 *
 *  ylt_dev     [n_layers][n_trials] FP64, values >= 0 (the YLT);
 *              1 <= n_trials <= 2^31 - 1, 1 <= n_layers <= 65535.
 *  probs_host  [n_p] probabilities in (0, 1); 1 <= n_p <= 8.
 *  mean_dev    [n_layers] FP64 output (may be NULL).
 *  pml_dev     [n_layers][n_p] FP64 output (may be NULL).
 *  tvar_dev    [n_layers][n_p] FP64 output (may be NULL).
 * Scratch is taken from the stream-ordered allocator and released on the
 * stream. Errors: ART_EINVAL, ART_ENOMEM, ART_ECUDA.
 */
ART_API art_status art_metrics(const double* ylt_dev, int64_t n_trials, int32_t n_layers, const double* probs_host,
                       int32_t n_p, double* mean_dev, double* pml_dev, double* tvar_dev, cudaStream_t stream);

/*
 * art_metrics_noalloc -- art_metrics without any device allocation. The
 * paper has no counterpart: this entry point exists for callers that must
 * not allocate device memory while they run. Examples are pricing services
 * that reserve all device memory up front under a fixed budget and treat
 * any later allocation as a failure, hosts whose device memory belongs to
 * another framework's allocator that must not be bypassed, and latency-
 * critical paths where an allocation's implicit synchronisation or its
 * failure modes are unacceptable.
 *
 * Same arguments, outputs and results as art_metrics. Instead of the
 * stream-ordered allocator it uses one scratch array that the library
 * defines in device memory at file scope, ART_METRICS_NOALLOC_SCRATCH_BYTES
 * (8 MiB) in size; every GPU that loads the library holds those 8 MiB until
 * the process exits. The fixed part of the scratch is about
 *   n_layers * 32.1 KiB + n_layers * n_p * 8.1 KiB
 * (a first-digit histogram per layer, a digit histogram per problem); a
 * call that needs more returns ART_EINVAL and enqueues nothing (in
 * practice, more than about 200 layers at one probability, 140 at three,
 * 80 at eight). What the fixed part leaves holds the candidate lists; a
 * layer whose list does not fit reads its whole row in every pass, which
 * gives the same results more slowly.
 *
 * The first call on each device looks up that device's address of the
 * scratch array (cudaGetSymbolAddress, with the device current); make that
 * first call before any stream capture. Every call on a device shares the
 * one array, and the array keeps the previous call's contents (each call
 * clears what must start at zero itself). Calls whose work overlaps on the
 * GPU -- on different streams, or from different threads -- race on the
 * scratch and give wrong results: order them on one stream or with events.
 * Calls no cudaMalloc, cudaFree or other allocating routine.
 */
#define ART_METRICS_NOALLOC_SCRATCH_BYTES (8u << 20)
ART_API art_status art_metrics_noalloc(const double* ylt_dev, int64_t n_trials, int32_t n_layers,
                                       const double* probs_host, int32_t n_p, double* mean_dev, double* pml_dev,
                                       double* tvar_dev, cudaStream_t stream);

/*
 * art_topk -- one shard's share of the metrics of a YLT split by trials
 * (Section III: trials are independent; Section IV-C: the multi-GPU runs
 * split the trials of the YET between the GPUs). PML_p and TVaR_p of a layer
 * depend only on its ceil((1 - p) N) largest trial losses, and those of the
 * whole YLT lie among the union of every shard's largest: per layer, this
 * writes the shard's k largest losses and its loss sum, and art_merge_topk
 * gives the whole YLT's metrics from the shards' outputs.
 *  ylt_dev   [n_layers][n_trials] FP64, this shard's trials (values >= 0);
 *            1 <= n_trials <= 2^31 - 1, 1 <= n_layers <= 65535.
 *  k         list length, 1 <= k <= 2^31 - 1.
 *  top_dev   [n_layers][k] FP64 output: the losses above the shard's
 *            min(k, n_trials)-th largest in trial order, then that loss as
 *            often as needed to fill min(k, n_trials) entries, then zeros.
 *  sum_dev   [n_layers] FP64 output (may be NULL): each layer's loss sum.
 * Deterministic (the same list for the same YLT). Scratch from the
 * stream-ordered allocator. Errors: ART_EINVAL, ART_ECUDA.
 */
ART_API art_status art_topk(const double* ylt_dev, int64_t n_trials, int32_t n_layers, int64_t k, double* top_dev,
                            double* sum_dev, cudaStream_t stream);

/*
 * art_merge_topk -- the merge step of sharded metrics (Section I: PML and
 * TVaR of the YLT; Section IV-C: trials split between GPUs), on the host.
 * From the lists and sums of n_shards shards (art_topk outputs gathered in
 * shard order), the mean, PML and TVaR of the whole YLT of n_trials_total
 * trials as art_metrics defines them: PML the k_q-th largest of the union of
 * the lists, k_q = ceil((1 - p_q) n_trials_total), TVaR the mean of the k_q
 * largest, the mean the shards' sums over n_trials_total.
 *  top_host   [n_shards][n_layers][k] FP64; sum_host [n_shards][n_layers] FP64.
 *  probs_host [n_p] in (0, 1), 1 <= n_p <= 8, every k_q <= k.
 *  mean_host  [n_layers], pml_host and tvar_host [n_layers][n_p]: host
 *             outputs, each may be NULL.
 * PML equals art_metrics on the whole YLT bit for bit; TVaR and the mean
 * differ only in the order of their FP64 additions (sums in shard and list
 * order: deterministic). Runs on host threads; needs no GPU.
 * Errors: ART_EINVAL (NULL inputs, sizes, probabilities, a k_q above k).
 */
ART_API art_status art_merge_topk(const double* top_host, const double* sum_host, int32_t n_shards, int32_t n_layers,
                                  int64_t k, int64_t n_trials_total, const double* probs_host, int32_t n_p,
                                  double* mean_host, double* pml_host, double* tvar_host);

/*
 * art_metrics_backward -- gradient of sum_j (gm_j mean_j + sum_q gt_{j,q}
 * TVaR_{j,q}) with respect to the YLT (the paper has no gradients; the
 * metrics are those of Section I, read as in art_metrics): grad_ylt[j][t] = gm_j / T
 * + sum_q gt_{j,q} w_{j,q}(t), where w = 1/k for Y > PML, (k - #greater) /
 * (k #equal) for Y == PML (ties share the boundary weight), 0 below.
 *  ylt_dev, n_trials, n_layers: as art_metrics; probs_host and n_p (0 <= n_p
 *                    <= 8) may be NULL and 0 when grad_tvar_dev is NULL.
 *  pml_dev           [n_layers][n_p] from art_metrics on the same YLT.
 *  grad_mean_dev     [n_layers] or NULL; grad_tvar_dev [n_layers][n_p] or NULL.
 *  grad_ylt_dev      [n_layers][n_trials] FP64 output.
 * Errors: ART_EINVAL (sizes, a NULL YLT or output, TVaR gradients without
 * PML or probabilities), ART_ENOMEM, ART_ECUDA.
 */
ART_API art_status art_metrics_backward(const double* ylt_dev, int64_t n_trials, int32_t n_layers,
                                const double* probs_host, int32_t n_p, const double* pml_dev,
                                const double* grad_mean_dev, const double* grad_tvar_dev,
                                double* grad_ylt_dev, cudaStream_t stream);

/*
 * art_run_ylt_backward -- adjoint of art_run_ylt (the paper has no
 * gradients; this is the pricing sensitivity). Given G = sum g_{j,t} Y_{j,t}:
 *   dG/dAggR_j = -sum_t g a,  dG/dAggL_j = sum_t g c,
 *   dG/dOccR_j = -sum_t g a #{d: OccR < x_d < OccR + OccL},
 *   dG/dOccL_j =  sum_t g a #{d: x_d > OccR + OccL},
 *   dG/dm_e    =  sum_j sum_t g a sum_d [o_d mid][D_e < m_e l < D_e + Lim_e] l,
 * with a = [branch == 1], c = [branch == 2] and l = l_e[E_{t,d}]; at a kink
 * the strict-inequality branch is taken. Trials whose branch is not 1 are not
 * re-read. The per-event branches are recomputed in FP32 as the forward
 * forms them; the results are deterministic.
 * With the ART_LAYOUT_GROUP tables the YET is read once per layer group and
 * only events with a loss in the group are evaluated; the per-event sums then
 * follow the group table's ELT order (the union of the group's layers' ELTs
 * in order of first appearance) and the
 * multiplier sums weight each event by g rounded to FP32, with compensated
 * FP32 accumulation (relative error of order 1e-7). Without them, the
 * ART_LAYOUT_LAYER tables are read once per layer in the layer's ELT order
 * (as the plain variant forms them) and g is applied in FP64 per trial.
 * An event whose per-event sum differs between the forward variant used and
 * this order can fall on the other side of an occurrence kink only when it
 * lies within FP32 rounding of that kink.
 *  branch_dev        [n_layers][T] from art_run_ylt on the same YET and terms.
 *  grad_ylt_dev      [n_layers][T] FP64.
 *  grad_terms_dev    [n_layers][4] FP64 output (OccR, OccL, AggR, AggL).
 *  grad_mult_dev     [n_elt] FP64 output.
 * Needs ART_LAYOUT_GROUP or ART_LAYOUT_LAYER (else ART_EUNSUPPORTED). Scratch
 * from the stream-ordered allocator.
 */
ART_API art_status art_run_ylt_backward(art_portfolio* p, int64_t n_trials, const int32_t* event_ids_dev,
                                const int64_t* trial_off_dev, int32_t events_per_trial,
                                const uint8_t* branch_dev, const double* grad_ylt_dev,
                                double* grad_terms_dev, double* grad_mult_dev, cudaStream_t stream);

/* Result of art_autotune. */
typedef struct {
    int32_t variant;      /* chosen ART_VARIANT_*                                  */
    int32_t slots;        /* layer tile of the persistent kernels: 32 * slots layers */
    int32_t trial_tile;   /* trials per work unit (0: the variant has none)        */
    int32_t cta_threads;  /* threads per CTA (0: the variant's fixed shape)        */
    float sample_ms;      /* best forward time on the sample                       */
    int32_t candidates;   /* shapes timed                                          */
    int32_t from_cache;   /* 1 when the shape came from the cache file             */
    int32_t mapping;      /* sparse variant: 0 event broadcast, 1 per-lane scatter  */
} art_tune_result;

/*
 * art_autotune -- pick the forward variant and the persistent kernels' tile
 * shapes (layer tile: 32, 64 or 128 layers per warp; trials per work unit
 * 1-16; 128 or 256 threads per CTA) by timing each candidate on the first
 * `sample_trials` trials (0: 65,536) of the given YET, and keep the one
 * whose time, extrapolated to n_trials, is least (as art_set_variant would
 * set it). When n_trials is at least twice the sample, each variant's
 * fastest shape is also timed on twice the sample, which separates the part
 * of a call that does not grow with the trials (such as the skip variant's
 * per-call occurrence tables) from the part that does; otherwise times
 * scale in proportion. ylt_dev is caller-owned scratch for the timed runs'
 * YLTs: [n_layers][min(n_trials, 2 * sample)] FP64. When the environment
 * variable ART_AUTOTUNE_CACHE names a file, a shape recorded there for the
 * same device, portfolio shape and YET shape (trials bucketed by powers of
 * two) is applied without timing, and a newly timed shape is appended.
 * Synchronises the stream. Not for use during stream capture. The paper
 * picks its threads per block by measurement too (Section IV); this widens
 * that to the variants and tile shapes here. Errors: ART_EINVAL,
 * ART_EUNSUPPORTED (no variant's layout was built), ART_ECUDA.
 */
ART_API art_status art_autotune(art_portfolio* p, int64_t n_trials, const int32_t* event_ids_dev,
                                const int64_t* trial_off_dev, int32_t events_per_trial, double* ylt_dev,
                                int32_t sample_trials, cudaStream_t stream, art_tune_result* out);

/* Synchronise the stream, then read and clear the portfolio's device error
 * flags: ART_OK, ART_EID_RANGE (an id outside [0, C) was seen; it counted as
 * zero loss: event ids index the direct-access tables of Section III) or
 * ART_EINVAL (decreasing CSR offsets were seen). Errors of the call itself:
 * ART_EINVAL (NULL portfolio), ART_ECUDA. */
ART_API art_status art_get_device_status(art_portfolio* p, cudaStream_t stream);

/* Bytes of device memory the portfolio holds, per layout (the direct-access
 * tables of Section III and their derived forms; NULL to skip). Errors:
 * ART_EINVAL (NULL portfolio). */
ART_API art_status art_get_footprint(const art_portfolio* p, int64_t* layer_bytes, int64_t* pool_bytes,
                                     int64_t* pool64_bytes, int64_t* group_bytes, int64_t* sparse_bytes);

/* Free the portfolio and every buffer it owns (synchronises the device
 * first). NULL is a no-op. No counterpart in the paper; never fails. */
ART_API void art_destroy_portfolio(art_portfolio* p);

/* Static, human-readable name of a status (an unknown code gets a generic
 * name). No counterpart in the paper; never fails. */
ART_API const char* art_status_string(art_status s);

/* Text of the last CUDA error this thread saw inside the library (empty
 * before any; the pointer stays valid until this thread's next library call
 * that records an error). No counterpart in the paper; never fails. */
ART_API const char* art_last_cuda_error(void);

/* Probe kinds for art_probe. */
enum {
    ART_PROBE_STREAM = 0,     /* streaming read of a buffer: GB/s of buffer bytes            */
    ART_PROBE_GATHER32 = 1,   /* random 32-byte sector reads: GB/s of sector bytes           */
    ART_PROBE_GATHER64 = 2,   /* random 64-byte row reads (two sectors): GB/s of row bytes   */
    ART_PROBE_GATHER4 = 3,    /* random 4-byte reads: GB/s of the 32-byte sectors touched    */
    ART_PROBE_FP64ADD = 4     /* independent FP64 adds: GFLOP/s                             */
};

/*
 * art_probe -- measure a limit the kernels run against (a measurement aid;
 * the paper has no counterpart). The random-read probes are the roofline
 * denominators of the table lookups of Section III: over a buffer below the
 * L2 size they measure the L2 gather rate, over one far above it the DRAM
 * gather rate. Allocates `bytes` (1 MiB .. 64 GiB; ignored for the FP64
 * probe) on the current device, runs one warm-up and `reps` timed launches on
 * the legacy default stream, writes the best rate to *result and frees the
 * buffer. Synchronous. Errors: ART_EINVAL, ART_ENOMEM, ART_ECUDA.
 */
ART_API art_status art_probe(int32_t kind, int64_t bytes, int32_t reps, double* result);

/* Library version, major * 10000 + minor * 100 + patch. No counterpart in
 * the paper; never fails. */
ART_API int32_t art_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ART_H */

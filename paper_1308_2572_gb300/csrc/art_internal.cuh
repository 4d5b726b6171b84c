// art_internal.cuh -- internal types and device helpers of libart.
//
// Everything here serves the kernels behind include/art.h. The method is
// Section II / Algorithm 1 of Bahl et al. (arXiv:1308.2572); the layouts are
// the direct-access tables of Section III, re-laid out event-major so that one
// event's losses across a layer's (or the pool's) ELTs are contiguous.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "art.h"

namespace art {

constexpr int kMaxLayerElts = 32;   // ELTs per layer (the paper: 3-30)
constexpr int kMaxPoolElts = 512;   // widest pool row the batched kernel reads
constexpr int kMaxProbs = 8;        // probabilities per art_metrics call

// Error flag slots in the portfolio's device flag array.
enum { kFlagIdRange = 0, kFlagBadOffsets = 1, kNumFlags = 4 };

// XL(v; R, L) = min(max(v - R, 0), L), the excess-of-loss form of the
// occurrence (Algorithm 1 step 3) and aggregate (step 4) terms.
__device__ __forceinline__ float xl_f32(float v, float r, float l) { return fminf(fmaxf(v - r, 0.0f), l); }
__device__ __forceinline__ double xl_f64(double v, double r, double l) { return fmin(fmax(v - r, 0.0), l); }

// Per-ELT financial terms (step 2), read as F(y) = XL(m y; D, Lim) with the
// product and the deductible in one FMA rounding.
__device__ __forceinline__ float fin_f32(float y, float m, float d, float lim) {
    return fminf(fmaxf(__fmaf_rn(m, y, -d), 0.0f), lim);
}
__device__ __forceinline__ double fin_f64(double y, double m, double d, double lim) {
    return fmin(fmax(fma(m, y, -d), 0.0), lim);
}

// Aggregate branch code stored for the adjoint: 1 strictly between the
// retention and retention + limit, 2 strictly above, 0 otherwise.
__device__ __forceinline__ uint8_t agg_branch(double s, double r, double l) {
    double w = s - r;
    if (!(w > 0.0)) return 0;
    if (w > l) return 2;
    if (w < l) return 1;
    return 0;
}

// Terms of one layer as the plain kernel reads them: passed by value, so they
// sit in the kernel-parameter constant bank and unrolled loops use them as
// constant operands. Padding ELTs (index >= n) have m = 1, D = 0, Lim = inf
// and zero table entries, so they add exactly 0.
struct LayerArgs {
    const float* table;   // [C][np] event-major direct-access table of the layer
    float m[kMaxLayerElts];
    float d[kMaxLayerElts];
    float lim[kMaxLayerElts];
    float occ_ret, occ_lim;
    double agg_ret, agg_lim;
    int32_t layer;        // layer index (row of the YLT)
};

struct YetArgs {
    const int32_t* ids;
    const int64_t* off;   // NULL: dense
    int64_t n_trials;
    int32_t k;            // events per trial when dense
    int32_t catalogue;
};

__device__ __forceinline__ void trial_range(const YetArgs& y, int64_t t, int64_t& b, int64_t& e, bool& bad) {
    if (y.off) {
        b = y.off[t];
        e = y.off[t + 1];
        bad = e < b;
        if (bad) e = b;
    } else {
        b = t * (int64_t)y.k;
        e = b + y.k;
        bad = false;
    }
}

// Streaming loads (evict-first) for the YET, read exactly once per pass.
__device__ __forceinline__ int32_t ld_stream(const int32_t* p) { return __ldcs(p); }

// Exact sums of non-negative FP64 values (the metrics' sums, the all-FP64
// forward's aggregates). A value's bit pattern (its "key") orders like the
// value; constexprs and helpers below work on keys.
constexpr unsigned long long kMant = (1ULL << 52) - 1;
constexpr int kFixBits = 44;  // fixed-point unit: 2^(e_ref - 1075 - kFixBits)

// Exponent of a fixed-point unit's reference: the largest key's binary
// exponent field (at least 1, the subnormals' scale).
__device__ __forceinline__ int ref_exp(unsigned long long kmax) { return max(1, (int)(kmax >> 52)); }

// A fixed-point sum: a 128-bit integer in units of 2^(e_ref - 1075 - kFixBits),
// e_ref the reference exponent of the summed values (that of the largest
// value that may occur). A key's mantissa shifted to its place is below
// 2^(53 + kFixBits), so 2^31 of them stay below 2^128. Bits below the unit
// are dropped: at most one unit, 2^-96 of the reference value, per term
// (the metrics' sums all hold the reference value itself; the all-FP64
// forward's aggregate sums at most a trial's events). Integer additions give
// the same bits in any order.
struct Fix {
    unsigned long long lo, hi;
};

// The key's value in those units as a mantissa m (< 2^53, already shifted
// down where the key lies below the unit's range) and a left shift sh
// (0 .. kFixBits). e_ref is at least the key's exponent.
__device__ __forceinline__ void fix_split(unsigned long long key, int e_ref, unsigned long long& m, int& sh) {
    const int e = (int)(key >> 52);
    m = (key & kMant) | (e ? (1ULL << 52) : 0ULL);
    sh = max(e, 1) - e_ref + kFixBits;  // <= kFixBits
    if (sh < 0) {
        m = -sh < 64 ? m >> -sh : 0ULL;
        sh = 0;
    }
}

// m * 2^sh as two words (sh <= kFixBits, m < 2^53).
__device__ __forceinline__ void fix_shift(unsigned long long m, int sh, unsigned long long& a0, unsigned long long& a1) {
    a0 = m << sh;
    a1 = sh > 11 ? m >> (64 - sh) : 0ULL;
}

// The key's value in those units as two words.
__device__ __forceinline__ void fix_words(unsigned long long key, int e_ref, unsigned long long& a0,
                                          unsigned long long& a1) {
    unsigned long long m;
    int sh;
    fix_split(key, e_ref, m, sh);
    fix_shift(m, sh, a0, a1);
}

// (m, sh) of fix_split in one word: m in bits 0-52, sh in bits 58-63; a
// value of 0 (m = 0) packs to 0, so packing a zero entry again keeps it 0.
// A table packed once per reference exponent spares each later add the
// split.
__device__ __forceinline__ unsigned long long fix_pack(unsigned long long key, int e_ref) {
    unsigned long long m;
    int sh;
    fix_split(key, e_ref, m, sh);
    return m ? m | ((unsigned long long)sh << 58) : 0ULL;
}

__device__ __forceinline__ void fix_add2(Fix& f, unsigned long long a0, unsigned long long a1) {
    f.lo += a0;
    f.hi += a1 + (f.lo < a0 ? 1ULL : 0ULL);
}

__device__ __forceinline__ void fix_add(Fix& f, unsigned long long key, int e_ref) {
    unsigned long long a0, a1;
    fix_words(key, e_ref, a0, a1);
    fix_add2(f, a0, a1);
}

// f += the value of a packed word (fix_pack): the same two words as fix_add
// of the key it was packed from.
__device__ __forceinline__ void fix_add_packed(Fix& f, unsigned long long w) {
    unsigned long long a0, a1;
    fix_shift(w & ((1ULL << 58) - 1), (int)(w >> 58), a0, a1);
    fix_add2(f, a0, a1);
}

// f += c * key (c < 2^32), exactly.
__device__ __forceinline__ void fix_add_times(Fix& f, unsigned long long key, int e_ref, unsigned long long c) {
    unsigned long long a0, a1;
    fix_words(key, e_ref, a0, a1);
    fix_add2(f, a0 * c, __umul64hi(a0, c) + a1 * c);
}

// Sum over the warp (valid in every lane).
__device__ __forceinline__ Fix fix_warp_sum(Fix f) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long b0 = __shfl_xor_sync(0xffffffffu, f.lo, o);
        const unsigned long long b1 = __shfl_xor_sync(0xffffffffu, f.hi, o);
        fix_add2(f, b0, b1);
    }
    return f;
}

// g[0..1] += f with integer atomics and the carry.
__device__ __forceinline__ void fix_atomic(unsigned long long* g, const Fix& f) {
    if (!(f.lo | f.hi)) return;
    const unsigned long long o0 = atomicAdd(g, f.lo);
    const unsigned long long hi = f.hi + (o0 + f.lo < o0 ? 1ULL : 0ULL);
    if (hi) atomicAdd(g + 1, hi);
}

// Block sum of a fixed-point value into g (one atomic pair per warp).
__device__ __forceinline__ void fix_block_atomic(unsigned long long* g, Fix f) {
    f = fix_warp_sum(f);
    if ((threadIdx.x & 31) == 0) fix_atomic(g, f);
}

// The FP64 value of a fixed-point sum. The scaling by the unit 2^n is one
// multiplication by 2^n (exact: t is an integer below 2^128, so the product
// is normal or overflows as scalbn's does) when 2^n is a normal double, else
// scalbn.
__device__ __forceinline__ double fix_value(const Fix& f, int e_ref) {
    const double t = fma((double)f.hi, 18446744073709551616.0, (double)f.lo);
    const int n = e_ref - 1075 - kFixBits;
    return n >= -1022 ? t * __longlong_as_double((long long)(n + 1023) << 52) : scalbn(t, n);
}

// Batched layout description shared by the host and the batched kernels.
struct BatchedArgs {
    const void* pool;          // [C][pool_np] FP32 or FP64
    const float* elt_terms;    // [3][pool_np]  m, D, Lim (FP32)
    const double* elt_terms64; // [3][pool_np]  same values in FP64
    const uint8_t* memb;       // [n_tiles][pool_np][32] slot bits per (ELT, lane)
    const int32_t* slot_layer; // [n_tiles][slots][32] layer of (slot, lane), -1 if empty
    const float* occ;          // [n_layers][2] OccR, OccL (FP32)
    const double* agg;         // [n_layers][2] AggR, AggL
    int32_t pool_np;
    int32_t n_layers;
    int32_t n_tiles;
    int32_t slots;
};

// One entry of the event-major CSR of the non-zero losses (ART_LAYOUT_SPARSE).
struct SparseEntry {
    float loss;
    int32_t elt;
};

// Compressed layout description (event-major CSR of the non-zero losses).
struct SparseArgs {
    const uint32_t* ptr;       // [C + 1]
    const void* entries;       // [nnz] (loss FP32, ELT int32)
    const float* elt_terms;    // [3][pool_np]
    const uint8_t* memb;       // [n_tiles][pool_np][32] slot bits per (ELT, lane)
    const uint16_t* tl_off;    // [n_tiles][pool_np + 1]: ELT e's layers in the tile are
    const uint8_t* tl_lay;     //   tl_lay[tile][tl_off[e] .. tl_off[e+1]) (tile-local index)
    const int32_t* slot_layer; // [n_tiles][slots][32]
    const float* occ;          // [n_layers][2]
    const double* agg;         // [n_layers][2]
    int32_t pool_np;
    int32_t n_tiles;
    int32_t tl_stride;         // bytes of tl_lay per tile (multiple of 16)
};

// A layer group for the bitmap-skip kernel: up to 8 layers whose ELTs number
// at most 32 together, with one event-major table over the union of those
// ELTs and an occupancy bitmap over the catalogue. Passed by value.
constexpr int kMaxGroupLayers = 8;
struct GroupArgs {
    const float* table;       // [C][np] FP32 over the group's ELTs (union order)
    const uint32_t* bitmap;   // [ceil(C / 32)]: bit i set if row i is not all zero
    float m[kMaxLayerElts];   // terms of the group's ELTs (padding: 1, 0, inf)
    float d[kMaxLayerElts];
    float lim[kMaxLayerElts];
    uint32_t member[kMaxGroupLayers];  // bit k: the group's ELT k belongs to the layer
    // the same membership as 0/1 coefficients: a layer's ELT sum is a chain of
    // FMAs x = fma(c, f, x), which rounds exactly as x + f (c = 1) or leaves x
    // unchanged (c = 0, f finite), with c a constant operand
    float coef[kMaxGroupLayers][kMaxLayerElts];
    float occ_ret[kMaxGroupLayers], occ_lim[kMaxGroupLayers];
    double agg_ret[kMaxGroupLayers], agg_lim[kMaxGroupLayers];
    int32_t layer[kMaxGroupLayers];
    int32_t n_layers;
};

// The skip variant works on occurrence groups: up to 8 consecutive layers,
// whatever their ELTs. Each forward call writes, per group, the
// occurrence-loss table X[i][s] = O_j(x_ij) for the group's layer j in slot s
// (Algorithm 1 steps 2-3 evaluated once per catalogue event; slots past the
// group's layers hold 0) and its bitmap (bit i set if any X[i][s] > 0); the
// trial pass then reads those. Passed by value.
constexpr int kMaxOccLayers = 8;
constexpr int kMaxOcc64Layers = 4;  // layers per FP64 occurrence group
struct OccGroupArgs {
    const float* occ;          // [C + 1][lt_pad] FP32
    const double* occ64;       // [C + 1][lt_pad] the all-FP64 tables (FP64, then packed fixed point)
    const unsigned long long* maxkey;  // the FP64 table's largest entry (its key), written by the build
    const uint32_t* occ_bits;  // bits 0 .. C, zero-padded to whole 16-byte groups
    int32_t layer[kMaxOccLayers];
    double agg_ret[kMaxOccLayers], agg_lim[kMaxOccLayers];
    int32_t n_layers;
};

// One layer as the occurrence-table build reads it (device array, one entry
// per layer; padding ELTs have m = 1, D = 0, Lim = inf and zero columns).
struct LayerBuildArgs {
    const float* table;        // the layer's [C][np] table (ART_LAYOUT_LAYER)
    float m[kMaxLayerElts];
    float d[kMaxLayerElts];
    float lim[kMaxLayerElts];
    float occ_ret, occ_lim;
    int32_t np;
    int32_t pad_;
};

// One occurrence group as the build reads it (device array).
struct OccBuildGroup {
    float* occ;
    uint32_t* occ_bits;
    unsigned long long* maxkey;  // FP64 groups: the table's largest entry (atomic maximum of keys)
    int32_t layer[kMaxOccLayers];
    int32_t n_layers;
    int32_t unsorted;            // skip groups: bit s set when layer s lists its ELTs out of ascending id order
};

}  // namespace art

// The opaque portfolio.
struct art_portfolio {
    int device = 0;
    int32_t catalogue = 0, n_elt = 0, n_layers = 0;
    int32_t layouts = 0, variant = ART_VARIANT_AUTO, flags = 0;
    int32_t trial_tile = 0, cta_threads = 0;
    int num_sms = 0;

    // terms as applied (after rounding)
    std::vector<float> mult, ded, lim, occ_ret, occ_lim;
    std::vector<double> agg_ret, agg_lim;
    std::vector<int32_t> loff, lids;

    // ART_LAYOUT_LAYER: per layer [C][np_j]
    std::vector<float*> layer_tab;
    std::vector<int32_t> layer_np;
    int64_t layer_bytes = 0;

    // ART_LAYOUT_POOL / POOL64: [C][pool_np]
    float* pool = nullptr;
    double* pool64 = nullptr;
    int32_t pool_np = 0;
    int64_t pool_bytes = 0, pool64_bytes = 0;

    // ART_LAYOUT_GROUP: layer groups with union tables and occupancy bitmaps
    std::vector<art::GroupArgs> groups;
    std::vector<int32_t> group_np;
    std::vector<std::vector<int32_t>> group_elts;   // union ELT ids per group
    std::vector<std::vector<int32_t>> group_layers; // layer ids per group
    std::vector<float*> group_tab;
    std::vector<uint32_t*> group_bitmap;

    // skip variant (needs ART_LAYOUT_LAYER): occurrence groups and their
    // per-call occurrence-loss tables and bitmaps
    std::vector<art::OccGroupArgs> ogroups;
    int32_t og_lp = 0;                          // slots per row of X (1, 2, 4 or 8)
    std::vector<float*> og_occ;
    std::vector<uint32_t*> og_bits;
    art::LayerBuildArgs* d_lbuild = nullptr;    // [n_layers]
    art::OccBuildGroup* d_ogroups = nullptr;    // [n_ogroups]
    int64_t occ_bytes = 0;
    // ART_LAYOUT_OCC64: the same groups with FP64 tables and their own bitmaps
    std::vector<art::OccGroupArgs> ogroups64;
    std::vector<double*> og_occ64;
    std::vector<uint32_t*> og_bits64;
    art::OccBuildGroup* d_ogroups64 = nullptr;  // bitmaps of the FP64 tables
    double** d_occ64_ptrs = nullptr;            // [n_ogroups64]
    unsigned long long* d_occ64_max = nullptr;  // [n_ogroups64]: each FP64 table's largest entry
    int32_t og_lp64 = 0;                        // slots per row of the FP64 tables (1, 2 or 4)
    uint8_t* d_slotmask = nullptr;              // [n_ogroups][pool_np]: slots of the skip group holding the ELT
    uint8_t* d_slotmask64 = nullptr;            // [n_ogroups64][pool_np]: slots of the group holding the ELT
    int64_t occ64_bytes = 0;
    int64_t group_bytes = 0;

    // ART_LAYOUT_SPARSE: event-major CSR of the non-zero losses
    uint32_t* sp_ptr = nullptr;
    void* sp_entries = nullptr;
    uint32_t sp_nnz = 0;
    int64_t sparse_bytes = 0;

    // batched metadata (device)
    float* d_elt_terms = nullptr;      // [3][pool_np]
    double* d_elt_terms64 = nullptr;   // [3][pool_np]
    uint8_t* d_memb = nullptr;
    int32_t* d_slot_layer = nullptr;
    uint16_t* d_tl_off = nullptr;      // per tile: ELT -> tile-local layer lists
    uint8_t* d_tl_lay = nullptr;
    int32_t tl_stride = 0;
    int32_t sparse_mapping = -1;       // 0 broadcast, 1 scatter, -1 by layer tile
    float* d_occ = nullptr;
    double* d_agg = nullptr;
    int32_t slots = 0, n_tiles = 0;
    unsigned int* d_work_counter = nullptr;

    int* d_flags = nullptr;            // [kNumFlags]
    int32_t* d_loff = nullptr;         // device copies of the layer lists
    int32_t* d_lids = nullptr;

    // host-run staging
    int32_t* stage_ids[2] = {nullptr, nullptr};
    int64_t* stage_off[2] = {nullptr, nullptr};
    double* stage_ylt[2] = {nullptr, nullptr};
    int64_t stage_ids_cap = 0, stage_trials_cap = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_done[2] = {nullptr, nullptr};
    // host-run path with metrics: the whole YLT and the metric outputs on the device
    double* host_ylt = nullptr;
    double* host_out = nullptr;
    int64_t host_ylt_cap = 0, host_out_cap = 0;
    void* host_scratch = nullptr;  // the metrics' scratch of that path
    size_t host_scratch_cap = 0;

    // cached graph of one batched launch
    cudaGraphExec_t graph_exec = nullptr;
    const void* graph_key[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t graph_key_n[2] = {0, 0};
};

namespace art {

// Host-side launchers (each returns a CUDA error code).
cudaError_t launch_plain(art_portfolio* p, const YetArgs& y, double* ylt, uint8_t* branch, cudaStream_t s);
cudaError_t launch_payouts(art_portfolio* p, int32_t j, const YetArgs& y, double* payouts, int32_t* exhaust,
                           double* ylt, cudaStream_t s);
cudaError_t launch_sparse(art_portfolio* p, const YetArgs& y, double* ylt, uint8_t* branch, cudaStream_t s);
cudaError_t build_sparse(art_portfolio* p, const float* src, cudaStream_t s);
// build: write the occurrence tables first (false: reuse the ones the last
// call on this stream wrote with the same terms)
cudaError_t launch_skip(art_portfolio* p, const YetArgs& y, double* ylt, uint8_t* branch, cudaStream_t s,
                        bool build = true);
cudaError_t launch_skip64(art_portfolio* p, const YetArgs& y, double* ylt, uint8_t* branch, cudaStream_t s,
                          bool build = true);
cudaError_t build_group_bitmap(const float* table, int32_t catalogue, int32_t np, uint32_t* bitmap, cudaStream_t s);
// Write every occurrence group's X and bitmap (one launch) from the layer tables.
cudaError_t build_occurrence(art_portfolio* p, cudaStream_t s);
cudaError_t launch_batched(art_portfolio* p, const YetArgs& y, double* ylt, uint8_t* branch, bool fp64,
                           cudaStream_t s);
cudaError_t launch_adjoint(art_portfolio* p, const YetArgs& y, const uint8_t* branch, const double* g,
                           double* grad_terms, double* grad_mult, cudaStream_t s);
cudaError_t launch_adjoint_groups(art_portfolio* p, const YetArgs& y, const uint8_t* branch, const double* g,
                                  double* grad_terms, double* grad_mult, cudaStream_t s);
// The metrics over scratch of at least metrics_scratch_bytes(...) bytes
// (scratch NULL or smaller: taken from the stream-ordered allocator and
// released on the stream).
cudaError_t metrics_run(const double* ylt, int64_t n, int32_t n_layers, const double* probs, int32_t n_p,
                        double* mean, double* pml, double* tvar, cudaStream_t s, void* scratch = nullptr,
                        size_t scratch_bytes = 0);
// The same with the ranks k given (clamped to [1, n]) instead of
// probabilities; sum_out (may be NULL) receives each layer's FP64 loss sum.
cudaError_t metrics_run_k(const double* ylt, int64_t n, int32_t n_layers, const int64_t* k, int32_t n_p,
                          double* mean, double* pml, double* tvar, double* sum_out, cudaStream_t s,
                          void* scratch = nullptr, size_t scratch_bytes = 0);
size_t metrics_scratch_bytes(int64_t n, int32_t n_layers, int32_t n_p);
cudaError_t metrics_backward_run(const double* ylt, int64_t n, int32_t n_layers, const double* probs,
                                 int32_t n_p, const double* pml, const double* gmean, const double* gtvar,
                                 double* gylt, cudaStream_t s);
cudaError_t build_layer_table(const float* src, int32_t catalogue, const int32_t* elts_dev, int32_t n,
                              int32_t np, float* dst, cudaStream_t s);
cudaError_t build_pool_table(const float* src, int32_t catalogue, int32_t n_elt, int32_t np, float* dst32,
                             double* dst64, cudaStream_t s);

// (Re)build the layer tile of the persistent kernels (slots layers per lane).
cudaError_t set_layer_tile(art_portfolio* p, int32_t slots);

// k = ceil((1 - p) N) with the integer guard; at least 1, at most N.
int64_t tail_count(double p, int64_t n);

void set_last_error(cudaError_t e);

// Set (bytes > 0) or clear (bytes == 0) a persisting L2 access-policy window
// over a hot table on a stream.
cudaError_t set_window(cudaStream_t s, const void* base, size_t bytes);

}  // namespace art

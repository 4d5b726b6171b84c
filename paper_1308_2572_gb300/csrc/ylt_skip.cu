// ylt_skip.cu -- the forward pass by occurrence groups with an occupancy
// bitmap (Section II, Algorithm 1, over Section III's direct-access tables,
// plus the occupancy summary that Section VI's compressed representations
// point to).
//
// Steps 2-3 of Algorithm 1 (the financial terms, the ELT sum and the
// occurrence terms) depend on the event id alone, not on the trial. So each
// call first evaluates them once per catalogue event, for every occurrence
// group (up to 8 consecutive layers): X[i][s] = O_j(sum_{e in layer j}
// F_e(l_e[i])) for the group's layer j in slot s, in FP32 and in the layer's
// ELT order (read from the per-layer tables), plus a bitmap with bit i set
// when any X[i][s] > 0. The trial pass then needs, per event occurrence, one
// bit test and, for the events with a non-zero occurrence loss, one gather
// of X[E_d] (4 * LP contiguous bytes); events with a clear bit add exactly 0
// to every layer and are skipped. The values are the ones the per-occurrence
// evaluation gives, bit for bit: the same operations on the same operands.
//
// Mapping of the trial pass: a persistent grid of one CTA per SM. Each CTA
// copies the bitmap into shared memory; when the catalogue's bits do not fit
// (227 KB hold 1.86M events), word w holds words w and w + S OR-ed together
// (a superset test: a fold-only hit gathers a row of zeros, which adds
// exactly 0), so the per-event test is always one shared-memory load for
// catalogues up to twice that. Each warp walks a strided sequence of trials
// as a stream of chunks of 32 * E events: the next chunk's ids (from the same
// trial or the next one) are requested before the current chunk is
// processed, hiding the DRAM latency of the id stream. Ids outside [0, C)
// map to the sentinel event C (bit clear, row zero); a per-lane maximum
// raises the range flag. For groups of 1-2 layers every lane gathers X for
// its own events whose bit is set (predicated loads, E in flight per lane).
// For wider groups the ids whose bit is set go to a per-warp
// queue in shared memory and each time 32 are queued every lane takes one,
// so the per-event work (one row of LP floats and LT accumulations) runs on
// full warps. The per-lane, per-layer aggregate is a compensated FP32 pair
// (Knuth's two-sum: the pair holds the exact sum up to a second-order term),
// and the warp reduces the lanes' pairs as compensated FP32 pairs too; the
// FP64 steps (the fold of the pair, the aggregate terms, the branch code)
// run once per 32 trials for groups of 1-2 layers (lane s keeps trial s) and
// on lane j for layer j otherwise, so the FP64 pipe is nearly idle.
#include <algorithm>
#include <limits>

#include "art_internal.cuh"

namespace art {

namespace {

#ifndef ART_SKIP_THREADS
#define ART_SKIP_THREADS 1024
#endif
#ifndef ART_SKIP_IDS_PER_LANE
#define ART_SKIP_IDS_PER_LANE 8
#endif
constexpr int kSkipThreads = ART_SKIP_THREADS;
constexpr int kSkipWarps = kSkipThreads / 32;
constexpr int kSkipIdsPerLane = ART_SKIP_IDS_PER_LANE;
constexpr int kQueue = 64;  // per-warp queue entries

__device__ __forceinline__ uint32_t ld_bitmap(const uint32_t* p) {
    uint32_t v;
    asm("ld.global.nc.L1::evict_last.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// 32 contiguous bytes of a row in one 256-bit load (sm_100 and later).
__device__ __forceinline__ void ld_row8(const float* p, float* v) {
    asm("ld.global.nc.L1::no_allocate.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
}

__device__ __forceinline__ void ld_row4(const float* p, float* v) {
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
        : "l"(p));
}

// s + e += v without losing the rounding error of the FP32 add (two-sum).
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float v) {
    const float t = s + v;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (v - bp);
    s = t;
    e += err;
}

__device__ __forceinline__ float ld_occ1(const float* p) {
    float v;
    asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void ld_occ2(const float* p, float* v) {
    asm("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v[0]), "=f"(v[1]) : "l"(p));
}

// Row i of the occurrence-loss table: LP (1, 2, 4 or 8) contiguous floats.
template <int LP>
__device__ __forceinline__ void ld_occ_row(const float* x, int32_t id, float (&o)[LP]) {
    const float* p = x + (size_t)id * LP;
    if constexpr (LP == 1) o[0] = ld_occ1(p);
    else if constexpr (LP == 2) ld_occ2(p, o);
    else if constexpr (LP == 4) ld_row4(p, o);
    else ld_row8(p, o);
}

// One row of X into the lane's per-layer pairs. Entries are >= 0 and a +0
// leaves a pair's bits unchanged under two-sum, so every slot is added
// without a test.
template <int LT>
__device__ __forceinline__ void add_occ(const float* o, float (&hi)[LT], float (&lo)[LT]) {
#pragma unroll
    for (int j = 0; j < LT; ++j) two_sum_acc(hi[j], lo[j], o[j]);
}

__device__ __forceinline__ int4 ld_stream4(const int32_t* p) {
    return __ldcs(reinterpret_cast<const int4*>(p));
}

// Position of id slot k of a lane within a chunk of 32 * E events starting at
// trial offset c0. Scalar layout: slot k is event c0 + 32 k + lane (each warp
// load is 128 contiguous bytes). Vector layout (trial start and length
// multiples of 4): slots 4h..4h+3 are events c0 + 128 h + 4 lane + 0..3, one
// 16-byte load.
template <bool VEC>
__device__ __forceinline__ int32_t slot_pos(int32_t c0, int k, int lane) {
    if constexpr (VEC) return c0 + 128 * (k >> 2) + 4 * lane + (k & 3);
    else return c0 + 32 * k + lane;
}

template <int E, bool VEC>
__device__ __forceinline__ void load_chunk(const int32_t* __restrict__ ids, int32_t c0, int32_t n, int lane,
                                           int32_t (&v)[E]) {
    if constexpr (VEC) {
#pragma unroll
        for (int h = 0; h < E / 4; ++h) {
            const int32_t d = c0 + 128 * h + 4 * lane;
            int4 w = make_int4(-1, -1, -1, -1);
            if (d < n) w = ld_stream4(ids + d);  // n and d are multiples of 4
            v[4 * h + 0] = w.x;
            v[4 * h + 1] = w.y;
            v[4 * h + 2] = w.z;
            v[4 * h + 3] = w.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int32_t d = c0 + 32 * k + lane;
            v[k] = d < n ? ld_stream(ids + d) : -1;
        }
    }
}

// True when every layer of the group has reached its aggregate cap: the sum
// of the lanes' partial aggregates is at least AggR + AggL. The aggregate
// never decreases (o >= 0), so the trial's loss is then AggL exactly.
template <int LT>
__device__ __forceinline__ bool group_capped(const OccGroupArgs& g, const float (&hi)[LT], const float (&lo)[LT]) {
    bool all = true;
#pragma unroll
    for (int j = 0; j < LT; ++j) {
        float v = hi[j] + lo[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (j < g.n_layers) all = all && ((double)v - g.agg_ret[j] >= g.agg_lim[j]);
    }
    return all;
}

// (h, l) += (h2, l2) for compensated FP32 pairs: two-sum of the high parts,
// the error and both low parts into the low part. Symmetric in its operands
// (the two-sum error is exact), so xor-shuffle reductions give every lane the
// same bits.
__device__ __forceinline__ void pair_add(float& h, float& l, float h2, float l2) {
    const float t = h + h2;
    const float bp = t - h;
    const float err = (h - (t - bp)) + (h2 - bp);
    h = t;
    l = (l + l2) + err;
}

template <int LT, int LP, bool VEC, bool COMPACT, bool FOLD>
__global__ void __launch_bounds__(kSkipThreads, 1) ylt_skip_kernel(const OccGroupArgs g, const YetArgs y,
                                                                  const int32_t smem_words, const bool early_exit,
                                                                  double* __restrict__ ylt,
                                                                  uint8_t* __restrict__ branch,
                                                                  int* __restrict__ flags) {
    constexpr unsigned FULL = 0xffffffffu;
    // ids per lane per chunk (a chunk is 32 * E events): the compacting
    // groups take 4, which leaves them registers without spills (c4 forward
    // 75.8 -> 65.1 ms with the untested adds below; the queue receives the
    // events in the same order, so the sums are the same bits)
    constexpr int E = COMPACT ? 4 : kSkipIdsPerLane;
    extern __shared__ __align__(16) uint32_t s_dyn[];
    int32_t* s_queue = reinterpret_cast<int32_t*>(s_dyn);  // [kSkipWarps][kQueue] (COMPACT only)
    uint32_t* s_bits = s_dyn + (COMPACT ? kSkipWarps * kQueue : 0);  // smem_words words of the bitmap
    {
        // FOLD: word w holds bitmap words w and w + smem_words OR-ed together
        // (a superset test: an event whose bit is set only through the fold
        // gathers a row of zeros, which adds exactly 0)
        const uint4* src = reinterpret_cast<const uint4*>(g.occ_bits);
        uint4* dst = reinterpret_cast<uint4*>(s_bits);
        const int words = (y.catalogue >> 5) + 1;  // bits 0 .. C (C: the sentinel)
        for (int i = threadIdx.x; i < smem_words / 4; i += blockDim.x) {
            uint4 v = src[i];
            if (FOLD && 4 * i + smem_words < words) {  // occ_bits is zero-padded to whole uint4
                const uint4 u = src[i + smem_words / 4];
                v.x |= u.x;
                v.y |= u.y;
                v.z |= u.z;
                v.w |= u.w;
            }
            dst[i] = v;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int32_t* q = s_queue + wib * kQueue;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n_warps = (int64_t)gridDim.x * kSkipWarps;
    uint32_t max_id = 0;  // largest id seen (an id >= C raises the range flag)
    bool bad_off_seen = false;

    // groups of 1-2 layers: results of up to 32 trials, lane s holding the
    // s-th, so the FP64 steps (fold of the pair, aggregate terms, branch code)
    // run once per 32 trials; wider groups: lane j finalises layer j of each
    // trial
    constexpr bool BATCH = LT <= 2;
    int32_t my_layer = 0;
    double my_ret = 0.0, my_lim = 0.0;
#pragma unroll
    for (int j = 0; j < LT; ++j)
        if (lane == j) {
            my_layer = g.layer[j];
            my_ret = g.agg_ret[j];
            my_lim = g.agg_lim[j];
        }
    float rh[BATCH ? LT : 1], rl[BATCH ? LT : 1];
    int64_t rt = -1;
    bool rcap = false;
    int slot = 0;
    auto flush = [&]() {
        if (BATCH && rt >= 0) {
#pragma unroll
            for (int j = 0; j < LT; ++j) {
                if (j < g.n_layers) {
                    const double sum = (double)rh[j] + (double)rl[j];
                    const size_t wi = (size_t)g.layer[j] * (size_t)y.n_trials + (size_t)rt;
                    // an early exit means every layer reached its cap: the loss is AggL
                    ylt[wi] = rcap ? g.agg_lim[j] : xl_f64(sum, g.agg_ret[j], g.agg_lim[j]);
                    if (branch) branch[wi] = rcap ? (uint8_t)2 : agg_branch(sum, g.agg_ret[j], g.agg_lim[j]);
                }
            }
        }
        rt = -1;
    };

    int64_t t = (int64_t)blockIdx.x * kSkipWarps + wib;
    const int32_t* tid = y.ids;  // ids of the current trial
    int32_t n = 0;               // its length
    int32_t pre[E];
    if (t < y.n_trials) {
        int64_t b, e;
        bool bo;
        trial_range(y, t, b, e, bo);
        bad_off_seen |= bo;
        tid = y.ids + b;
        n = (int32_t)(e - b);
        load_chunk<E, VEC>(tid, 0, n, lane, pre);
    }
    while (t < y.n_trials) {
        const int64_t tn = t + n_warps;
        const int32_t* tidn = y.ids;
        int32_t nn = 0;
        if (tn < y.n_trials) {
            int64_t bn, en;
            bool bo;
            trial_range(y, tn, bn, en, bo);
            bad_off_seen |= bo;
            tidn = y.ids + bn;
            nn = (int32_t)(en - bn);
        }
        float hi[LT], lo[LT];
#pragma unroll
        for (int j = 0; j < LT; ++j) {
            hi[j] = 0.0f;
            lo[j] = 0.0f;
        }
        int qn = 0;  // warp-uniform queue length, < 32 between steps
        bool capped_exit = false;
        if (n == 0 && tn < y.n_trials) load_chunk<E, VEC>(tidn, 0, nn, lane, pre);
        for (int32_t c0 = 0; c0 < n; c0 += 32 * E) {
            int32_t id[E];
#pragma unroll
            for (int k = 0; k < E; ++k) id[k] = pre[k];
            const bool full_chunk = c0 + 32 * E <= n;
            // request the next chunk (this trial's, or the next trial's first) now
            if (c0 + 32 * E < n) load_chunk<E, VEC>(tid, c0 + 32 * E, n, lane, pre);
            else if (tn < y.n_trials) load_chunk<E, VEC>(tidn, 0, nn, lane, pre);
            // ids outside [0, C) (and the empty slots of a partial chunk) map
            // to the sentinel C: its bit is clear and its row of X is zero
            uint32_t uid[E];
            if (full_chunk) {  // every slot of a full chunk is an event of the trial
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    max_id = max(max_id, (uint32_t)id[k]);
                    uid[k] = min((uint32_t)id[k], (uint32_t)y.catalogue);
                }
            } else {
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const bool live = slot_pos<VEC>(c0, k, lane) < n;
                    max_id = max(max_id, live ? (uint32_t)id[k] : 0u);
                    uid[k] = live ? min((uint32_t)id[k], (uint32_t)y.catalogue) : (uint32_t)y.catalogue;
                }
            }
            bool nz[E];
#pragma unroll
            for (int k = 0; k < E; ++k) {
                uint32_t wi = uid[k] >> 5;
                uint32_t w;
                if constexpr (FOLD) {
                    wi = min(wi, wi - (uint32_t)smem_words);  // wi - S wraps when wi < S
                    w = s_bits[wi];
                } else {
                    w = wi < (uint32_t)smem_words ? s_bits[wi] : ld_bitmap(g.occ_bits + wi);
                }
                nz[k] = __funnelshift_r(w, 0u, uid[k]) & 1u;  // bit uid mod 32 of the word
            }
            if constexpr (COMPACT) {
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const unsigned m = __ballot_sync(FULL, nz[k]);
                    if (nz[k]) q[qn + __popc(m & lt_mask)] = (int32_t)uid[k];
                    qn += __popc(m);
                    if (qn >= 32) {
                        __syncwarp();
                        const int32_t mine = q[lane];
                        const int32_t carry = q[32 + lane];
                        __syncwarp();
                        q[lane] = carry;  // entries 32 .. qn-1 move to the front
                        qn -= 32;
                        float o[LP];
                        ld_occ_row<LP>(g.occ, mine, o);
                        add_occ<LT>(o, hi, lo);
                        __syncwarp();
                    }
                }
            } else {
                // every lane gathers its own non-zero events, E loads in flight
                float o[E][LP];
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    if (nz[k]) ld_occ_row<LP>(g.occ, (int32_t)uid[k], o[k]);
                    else {
#pragma unroll
                        for (int j = 0; j < LP; ++j) o[k][j] = 0.0f;
                    }
                }
#pragma unroll
                // empty slots hold +0, which two-sum adds exactly: no test
#pragma unroll
                for (int k = 0; k < E; ++k)
#pragma unroll
                    for (int j = 0; j < LT; ++j) two_sum_acc(hi[j], lo[j], o[k][j]);
            }
            if (early_exit && group_capped<LT>(g, hi, lo)) {
                // the rest of the trial cannot change its loss: skip it (and
                // the queued events); request the next trial's first chunk
                if (c0 + 32 * E < n && tn < y.n_trials) load_chunk<E, VEC>(tidn, 0, nn, lane, pre);
                qn = 0;
                capped_exit = true;
                break;
            }
        }
        if constexpr (COMPACT) {
            __syncwarp();
            if (lane < qn) {
                float o[LP];
                ld_occ_row<LP>(g.occ, q[lane], o);
                add_occ<LT>(o, hi, lo);
            }
            __syncwarp();
        }
        // the trial's aggregate: the lanes' pairs summed across the warp in
        // compensated FP32
#pragma unroll
        for (int j = 0; j < LT; ++j) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
                pair_add(hi[j], lo[j], __shfl_xor_sync(FULL, hi[j], o), __shfl_xor_sync(FULL, lo[j], o));
        }
        if constexpr (BATCH) {
            if (lane == slot) {
#pragma unroll
                for (int j = 0; j < LT; ++j) {
                    rh[j] = hi[j];
                    rl[j] = lo[j];
                }
                rt = t;
                rcap = capped_exit;
            }
            if (++slot == 32) {
                flush();
                slot = 0;
            }
        } else {
            float mh = 0.0f, ml = 0.0f;
#pragma unroll
            for (int j = 0; j < LT; ++j)
                if (lane == j) {
                    mh = hi[j];
                    ml = lo[j];
                }
            if (lane < g.n_layers) {
                const double sum = (double)mh + (double)ml;
                const size_t wi = (size_t)my_layer * (size_t)y.n_trials + (size_t)t;
                ylt[wi] = capped_exit ? my_lim : xl_f64(sum, my_ret, my_lim);
                if (branch) branch[wi] = capped_exit ? (uint8_t)2 : agg_branch(sum, my_ret, my_lim);
            }
        }
        t = tn;
        tid = tidn;
        n = nn;
    }
    flush();
    if (max_id >= (uint32_t)y.catalogue) atomicOr(flags + kFlagIdRange, 1);
    if (lane == 0 && bad_off_seen) atomicOr(flags + kFlagBadOffsets, 1);
}

// Occurrence-loss tables (steps 2-3 once per catalogue event): block
// (x, y) covers 256 events of occurrence group y; thread i sums F_e over row
// i of each of the group's layer tables in the layer's ELT order (padding
// columns add exactly 0), applies the occurrence terms and writes X[i][0..LP)
// (slots past the group's layers: 0); lane 0 of each warp writes the bitmap
// word of its 32 events. The group's layer terms are staged in shared memory.
template <int LP>
__global__ void __launch_bounds__(256) build_occ_kernel(const LayerBuildArgs* __restrict__ lbuild,
                                                        const OccBuildGroup* __restrict__ groups, int32_t catalogue,
                                                        int32_t words) {
    __shared__ LayerBuildArgs s_lb[LP];
    const OccBuildGroup& grp = groups[blockIdx.y];
    const int nl = grp.n_layers;
    for (int w = threadIdx.x; w < nl * (int)(sizeof(LayerBuildArgs) / 4); w += blockDim.x) {
        const int s = w / (int)(sizeof(LayerBuildArgs) / 4), o = w % (int)(sizeof(LayerBuildArgs) / 4);
        reinterpret_cast<uint32_t*>(&s_lb[s])[o] = reinterpret_cast<const uint32_t*>(&lbuild[grp.layer[s]])[o];
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool nz = false;
    if (i < catalogue) {
        float o[LP];
#pragma unroll
        for (int s = 0; s < LP; ++s) {
            o[s] = 0.0f;
            if (s < nl) {
                const LayerBuildArgs& a = s_lb[s];
                const int nq = a.np / 4;
                const float4* row = reinterpret_cast<const float4*>(a.table) + i * nq;
                // every 16-byte piece of the row requested at once, then
                // summed in ELT order
                float4 r[kMaxLayerElts / 4];
#pragma unroll
                for (int q = 0; q < kMaxLayerElts / 4; ++q)
                    r[q] = q < nq ? __ldcs(row + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                float x = 0.0f;
#pragma unroll
                for (int q = 0; q < kMaxLayerElts / 4; ++q) {
                    if (q < nq) {
                        x += fin_f32(r[q].x, a.m[4 * q + 0], a.d[4 * q + 0], a.lim[4 * q + 0]);
                        x += fin_f32(r[q].y, a.m[4 * q + 1], a.d[4 * q + 1], a.lim[4 * q + 1]);
                        x += fin_f32(r[q].z, a.m[4 * q + 2], a.d[4 * q + 2], a.lim[4 * q + 2]);
                        x += fin_f32(r[q].w, a.m[4 * q + 3], a.d[4 * q + 3], a.lim[4 * q + 3]);
                    }
                }
                o[s] = xl_f32(x, a.occ_ret, a.occ_lim);
                nz |= o[s] > 0.0f;
            }
        }
        float* dst = grp.occ + i * LP;
        if constexpr (LP == 1) dst[0] = o[0];
        else if constexpr (LP == 2) *reinterpret_cast<float2*>(dst) = make_float2(o[0], o[1]);
        else {
#pragma unroll
            for (int q = 0; q < LP / 4; ++q)
                reinterpret_cast<float4*>(dst)[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, nz);
    if ((threadIdx.x & 31) == 0 && (i >> 5) < words) grp.occ_bits[i >> 5] = m;
}

// The same tables from the event-major CSR of the non-zero losses: thread i
// walks event i's entries (in ELT id order) and adds F_e in FP32 to the
// slots of the group's layers that hold ELT e. For a layer that lists its
// ELTs in ascending id order that is the layer's own order, and the absent
// losses, zeros, would add exactly 0, so the sum is the per-layer build's
// bit for bit. For a layer listed out of order the same holds while the
// event has at most two of its entries (one or two terms give the same bits
// in either order); with three or more the thread re-sums that layer from
// its per-layer row, in the layer's order, as the per-layer build does.
template <int LP>
__global__ void __launch_bounds__(256) build_occ_csr_kernel(const uint32_t* __restrict__ ptr,
                                                            const SparseEntry* __restrict__ entries,
                                                            const float* __restrict__ terms, int32_t np,
                                                            const uint8_t* __restrict__ slotmask,
                                                            const float* __restrict__ occ_terms,
                                                            const LayerBuildArgs* __restrict__ lbuild,
                                                            const OccBuildGroup* __restrict__ groups, int32_t catalogue,
                                                            int32_t words) {
    const OccBuildGroup& grp = groups[blockIdx.y];
    const uint8_t* sm = slotmask + (size_t)blockIdx.y * np;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool nz = false;
    if (i < catalogue) {
        const int unsorted = grp.unsorted;
        float x[LP];
        int cnt[LP];
#pragma unroll
        for (int s = 0; s < LP; ++s) {
            x[s] = 0.0f;
            cnt[s] = 0;
        }
        const uint32_t k1 = ptr[i + 1];
        for (uint32_t k = ptr[i]; k < k1; ++k) {
            const SparseEntry en = entries[k];
            const uint32_t mask = sm[en.elt];
            if (!mask) continue;
            const float f = fin_f32(en.loss, terms[en.elt], terms[np + en.elt], terms[2 * np + en.elt]);
#pragma unroll
            for (int s = 0; s < LP; ++s)
                if ((mask >> s) & 1u) {
                    x[s] += f;
                    ++cnt[s];
                }
        }
        float o[LP];
#pragma unroll
        for (int s = 0; s < LP; ++s) {
            o[s] = 0.0f;
            if (s < grp.n_layers) {
                const int32_t j = grp.layer[s];
                if (((unsorted >> s) & 1) && cnt[s] >= 3) {
                    const LayerBuildArgs& a = lbuild[j];
                    const float* row = a.table + i * a.np;
                    float xs = 0.0f;
                    for (int c = 0; c < a.np; ++c) xs += fin_f32(row[c], a.m[c], a.d[c], a.lim[c]);
                    x[s] = xs;
                }
                o[s] = xl_f32(x[s], occ_terms[2 * j], occ_terms[2 * j + 1]);
                nz |= o[s] > 0.0f;
            }
        }
        float* dst = grp.occ + i * LP;
        if constexpr (LP == 1) dst[0] = o[0];
        else if constexpr (LP == 2) *reinterpret_cast<float2*>(dst) = make_float2(o[0], o[1]);
        else {
#pragma unroll
            for (int q = 0; q < LP / 4; ++q)
                reinterpret_cast<float4*>(dst)[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
        }
    }
    const unsigned m = __ballot_sync(0xffffffffu, nz);
    if ((threadIdx.x & 31) == 0 && (i >> 5) < words) grp.occ_bits[i >> 5] = m;
}

template <int LT, int LP>
cudaError_t launch_group(const OccGroupArgs& g, const YetArgs& y, int num_sms, int32_t catalogue, bool early,
                         double* ylt, uint8_t* branch, int* flags, cudaStream_t s) {
    constexpr bool COMPACT = LT >= 4;
    int dev = 0, max_optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
    const int queue_bytes = COMPACT ? kSkipWarps * kQueue * 4 : 0;
    const int words = (catalogue >> 5) + 1;  // bits 0 .. C (C: the sentinel)
    // whole 16-byte groups of words that fit next to the queues
    const int smem_words = std::max(4, std::min((words + 3) & ~3, (max_optin - queue_bytes) / 4) & ~3);
    const int smem = queue_bytes + smem_words * 4;
    // the bitmap folds once into shared memory when it is at most twice as long
    const bool fold = words <= 2 * smem_words;
    // 16-byte id loads when every trial starts and ends on a multiple of 4 ids
    const bool vec = !y.off && y.k % 4 == 0 && (reinterpret_cast<uintptr_t>(y.ids) & 15) == 0;
    auto kern = vec ? (fold ? ylt_skip_kernel<LT, LP, true, COMPACT, true> : ylt_skip_kernel<LT, LP, true, COMPACT, false>)
                    : (fold ? ylt_skip_kernel<LT, LP, false, COMPACT, true> : ylt_skip_kernel<LT, LP, false, COMPACT, false>);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    const int64_t grid = std::min<int64_t>(num_sms, (y.n_trials + kSkipWarps - 1) / kSkipWarps);
    kern<<<(unsigned)std::max<int64_t>(1, grid), kSkipThreads, smem, s>>>(g, y, smem_words, early, ylt, branch,
                                                                          flags);
    return cudaGetLastError();
}

// Bitmap of a group table: bit i set when row i has any non-zero entry.
__global__ void build_bitmap_kernel(const float* __restrict__ table, int32_t catalogue, int32_t np,
                                    uint32_t* __restrict__ bitmap) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool nz = false;
    if (i < catalogue)
        for (int k = 0; k < np; ++k) nz |= table[i * np + k] != 0.0f;
    const unsigned m = __ballot_sync(0xffffffffu, nz);
    if ((threadIdx.x & 31) == 0 && i < catalogue) bitmap[i >> 5] = m;
}

}  // namespace

cudaError_t build_group_bitmap(const float* table, int32_t catalogue, int32_t np, uint32_t* bitmap, cudaStream_t s) {
    const int64_t n = ((int64_t)catalogue + 31) / 32 * 32;
    build_bitmap_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(table, catalogue, np, bitmap);
    return cudaGetLastError();
}

cudaError_t build_occurrence(art_portfolio* p, cudaStream_t s) {
    const int32_t words = (int32_t)(((int64_t)p->catalogue + 31) / 32);
    const dim3 grid((unsigned)(((int64_t)words * 32 + 255) / 256), (unsigned)p->ogroups.size());
    // from the CSR of the non-zero losses where the portfolio holds it (see
    // build_occ_csr_kernel)
    if (p->d_slotmask && p->sp_ptr && p->d_elt_terms && p->d_occ && p->d_lbuild) {
        const SparseEntry* en = reinterpret_cast<const SparseEntry*>(p->sp_entries);
        switch (p->og_lp) {
            case 1: build_occ_csr_kernel<1><<<grid, 256, 0, s>>>(p->sp_ptr, en, p->d_elt_terms, p->pool_np, p->d_slotmask, p->d_occ, p->d_lbuild, p->d_ogroups, p->catalogue, words); break;
            case 2: build_occ_csr_kernel<2><<<grid, 256, 0, s>>>(p->sp_ptr, en, p->d_elt_terms, p->pool_np, p->d_slotmask, p->d_occ, p->d_lbuild, p->d_ogroups, p->catalogue, words); break;
            case 4: build_occ_csr_kernel<4><<<grid, 256, 0, s>>>(p->sp_ptr, en, p->d_elt_terms, p->pool_np, p->d_slotmask, p->d_occ, p->d_lbuild, p->d_ogroups, p->catalogue, words); break;
            case 8: build_occ_csr_kernel<8><<<grid, 256, 0, s>>>(p->sp_ptr, en, p->d_elt_terms, p->pool_np, p->d_slotmask, p->d_occ, p->d_lbuild, p->d_ogroups, p->catalogue, words); break;
            default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (p->og_lp) {
        case 1: build_occ_kernel<1><<<grid, 256, 0, s>>>(p->d_lbuild, p->d_ogroups, p->catalogue, words); break;
        case 2: build_occ_kernel<2><<<grid, 256, 0, s>>>(p->d_lbuild, p->d_ogroups, p->catalogue, words); break;
        case 4: build_occ_kernel<4><<<grid, 256, 0, s>>>(p->d_lbuild, p->d_ogroups, p->catalogue, words); break;
        case 8: build_occ_kernel<8><<<grid, 256, 0, s>>>(p->d_lbuild, p->d_ogroups, p->catalogue, words); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_skip(art_portfolio* p, const YetArgs& y, double* ylt, uint8_t* branch, cudaStream_t s,
                        bool build) {
    const bool early = (p->flags & ART_FLAG_EARLY_EXIT) != 0;
    // steps 2-3 once per catalogue event, with the terms as they are now
    cudaError_t err = build ? build_occurrence(p, s) : cudaSuccess;
    if (err != cudaSuccess || y.n_trials == 0) return err;
    // ART_FLAG_L2_PERSIST: a persisting window over the table each group
    // pass gathers from, so that the id stream does not evict it
    const bool window = (p->flags & ART_FLAG_L2_PERSIST) != 0;
    const size_t table_bytes = sizeof(float) * ((size_t)p->catalogue + 1) * (size_t)p->og_lp;
    for (const OccGroupArgs& g : p->ogroups) {
        if (window && (err = set_window(s, g.occ, table_bytes))) return err;
        switch (p->og_lp) {
            case 1: err = launch_group<1, 1>(g, y, p->num_sms, p->catalogue, early, ylt, branch, p->d_flags, s); break;
            case 2: err = launch_group<2, 2>(g, y, p->num_sms, p->catalogue, early, ylt, branch, p->d_flags, s); break;
            case 4: err = launch_group<4, 4>(g, y, p->num_sms, p->catalogue, early, ylt, branch, p->d_flags, s); break;
            case 8: err = launch_group<8, 8>(g, y, p->num_sms, p->catalogue, early, ylt, branch, p->d_flags, s); break;
            default: err = cudaErrorInvalidValue;
        }
        if (err != cudaSuccess) return err;
    }
    return window ? set_window(s, nullptr, 0) : cudaSuccess;
}

}  // namespace art

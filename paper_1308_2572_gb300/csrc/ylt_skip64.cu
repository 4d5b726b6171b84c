// ylt_skip64.cu -- the all-FP64 forward over occurrence tables (Section II,
// Algorithm 1), for the precision study: every step in FP64.
//
// As in the skip variant, steps 2-3 (financial terms, ELT sum, occurrence
// terms) depend on the event id alone, so each call evaluates them once per
// catalogue event, here in FP64: X[i][s] = O_j(sum_{e in layer j} F_e(l_e[i]))
// for the layer j in slot s of each FP64 occurrence group (up to 4
// consecutive layers, so that a group's table stays in L2), with F_e(y) =
// min(max(m_e y - D_e, 0), Lim_e) as one FP64 FMA and the terms (stored
// rounded to FP32) widened exactly. With the CSR of the non-zero losses
// (ART_LAYOUT_SPARSE) the tables are built from it: per event, F_e of each
// non-zero loss once, added to the slots of the layers holding ELT e, each
// layer's sum in ELT id order, so the FP64 work scales with the non-zero
// losses. Otherwise they come from the per-layer tables (the layer's ELT
// order; rows without losses give x = 0, o = 0 and skip the arithmetic). A
// bitmap marks the events with some X[i][s] > 0 (bit C, the sentinel for ids
// outside [0, C), is clear and row C is zero).
//
// The trial pass: a persistent grid of one 1024-thread CTA per SM, the bitmap
// in shared memory (folded once when it does not fit: a superset test, a
// fold-only hit gathers a zero row), a warp per trial streaming its ids with
// the next chunk requested before the current one is processed, and a
// per-warp queue of the events whose bit is set, evaluated 32 at a time (lane
// = event): one row of X (8 * LP bytes) added to the lane's per-layer sums.
// The sums are exact: each FP64 occurrence loss is added as an integer to a
// 128-bit fixed-point number whose unit is 2^-96 of the group table's largest
// entry (the build records it), so the aggregate S is the exact sum of the
// trial's FP64 occurrence losses up to one unit per event, rounded to FP64
// once. After the build each table entry is packed in place into the
// mantissa and shift of its fixed-point value, so a pass adds an entry with
// two shifts and a 128-bit add. The lanes' sums are reduced across the warp
// (xor shuffles: every lane holds every layer's total) and lane j applies
// layer j's aggregate terms in FP64. Integer adds replace the FP64 adds of a sequential sum, of which this
// part has about 0.53 TFLOP/s.
#include <algorithm>
#include <limits>

#include "art_internal.cuh"

namespace art {

namespace {

constexpr int k64Threads = 1024;
constexpr int k64Warps = k64Threads / 32;
constexpr int k64Ids = 4;     // ids per lane per chunk (no register spills; c4 137.5 -> 128.2 ms)
constexpr int k64Queue = 64;  // per-warp queue entries

__device__ __forceinline__ uint32_t ld_bits_global(const uint32_t* p) {
    uint32_t v;
    asm("ld.global.nc.L1::evict_last.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// The table's largest entry: a warp maximum of the keys, one atomic per warp.
__device__ __forceinline__ void note_max(unsigned long long* maxkey, unsigned long long mk) {
    for (int o = 16; o > 0; o >>= 1) mk = max(mk, __shfl_xor_sync(0xffffffffu, mk, o));
    if ((threadIdx.x & 31) == 0 && mk) atomicMax(maxkey, mk);
}

// Row id of X: its LP FP64 entries as bit patterns, in one load of 8 * LP
// bytes (a 32-byte row in one 256-bit load), not kept in L1. The table of
// each group is its own allocation, so row id starts on an 8 * LP-byte
// boundary. (Two 16-byte loads of FP64-typed registers per row made the
// pass 3.6 times slower: c4, 627 against 173 ms.)
template <int LP>
__device__ __forceinline__ void ld_row64(const double* x, uint32_t id, unsigned long long (&o)[LP]) {
    static_assert(LP == 1 || LP == 2 || LP == 4, "FP64 groups hold 1, 2 or 4 layers");
    const double* p = x + (size_t)id * LP;
    if constexpr (LP == 1) {
        asm("ld.global.nc.L1::no_allocate.u64 %0, [%1];" : "=l"(o[0]) : "l"(p));
    } else if constexpr (LP == 2) {
        asm("ld.global.nc.L1::no_allocate.v2.u64 {%0, %1}, [%2];" : "=l"(o[0]), "=l"(o[1]) : "l"(p));
    } else {
        asm("ld.global.nc.L1::no_allocate.v4.u64 {%0, %1, %2, %3}, [%4];"
            : "=l"(o[0]), "=l"(o[1]), "=l"(o[2]), "=l"(o[3])
            : "l"(p));
    }
}

// Block (x, y): 256 events of occurrence group y; thread i reads row i of
// each of the group's layer tables and writes X[i][0..LP) in FP64.
template <int LP>
__global__ void __launch_bounds__(256) build_occ64_kernel(const LayerBuildArgs* __restrict__ lbuild,
                                                          const OccBuildGroup* __restrict__ groups,
                                                          double* const* __restrict__ occ64, int32_t catalogue,
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
    unsigned long long mk = 0;  // the largest entry this thread writes (its key: entries are >= 0)
    if (i < catalogue) {
        double o[LP];
#pragma unroll
        for (int s = 0; s < LP; ++s) {
            o[s] = 0.0;
            if (s < nl) {
                const LayerBuildArgs& a = s_lb[s];
                const int nq = a.np / 4;
                const float4* row = reinterpret_cast<const float4*>(a.table) + i * nq;
                float4 r[kMaxLayerElts / 4];
#pragma unroll
                for (int q = 0; q < kMaxLayerElts / 4; ++q)
                    r[q] = q < nq ? __ldcs(row + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                // a row without losses gives x = 0 (F(0) = 0: D >= 0) and
                // o = 0 (OccR >= 0): its FP64 arithmetic is skipped
                bool any = false;
#pragma unroll
                for (int q = 0; q < kMaxLayerElts / 4; ++q)
                    any |= (r[q].x != 0.0f) | (r[q].y != 0.0f) | (r[q].z != 0.0f) | (r[q].w != 0.0f);
                if (!any) continue;
                double x = 0.0;
#pragma unroll
                for (int q = 0; q < kMaxLayerElts / 4; ++q) {
                    if (q < nq) {
                        x += fin_f64(r[q].x, a.m[4 * q + 0], a.d[4 * q + 0], a.lim[4 * q + 0]);
                        x += fin_f64(r[q].y, a.m[4 * q + 1], a.d[4 * q + 1], a.lim[4 * q + 1]);
                        x += fin_f64(r[q].z, a.m[4 * q + 2], a.d[4 * q + 2], a.lim[4 * q + 2]);
                        x += fin_f64(r[q].w, a.m[4 * q + 3], a.d[4 * q + 3], a.lim[4 * q + 3]);
                    }
                }
                o[s] = xl_f64(x, a.occ_ret, a.occ_lim);
                nz |= o[s] > 0.0;
            }
        }
        double* dst = occ64[blockIdx.y] + i * LP;
        if constexpr (LP == 1) dst[0] = o[0];
        else {
#pragma unroll
            for (int q = 0; q < LP / 2; ++q) reinterpret_cast<double2*>(dst)[q] = make_double2(o[2 * q], o[2 * q + 1]);
        }
#pragma unroll
        for (int s = 0; s < LP; ++s) mk = max(mk, (unsigned long long)__double_as_longlong(o[s]));
    }
    note_max(grp.maxkey, mk);
    const unsigned m = __ballot_sync(0xffffffffu, nz);
    if ((threadIdx.x & 31) == 0 && (i >> 5) < words) grp.occ_bits[i >> 5] = m;
}

// The same tables from the event-major CSR of the non-zero losses: thread i
// walks event i's entries (in ELT order) and adds F_e in FP64 to the slots of
// the group's layers that hold ELT e (a per-group mask per ELT). Only the
// events' non-zero losses are touched, so the FP64 work is per non-zero loss
// rather than per table column; each layer's sum follows ELT id order.
template <int LP>
__global__ void __launch_bounds__(256) build_occ64_csr_kernel(const uint32_t* __restrict__ ptr,
                                                              const SparseEntry* __restrict__ entries,
                                                              const double* __restrict__ terms64, int32_t np,
                                                              const uint8_t* __restrict__ slotmask,
                                                              const float* __restrict__ occ_terms,
                                                              const OccBuildGroup* __restrict__ groups,
                                                              double* const* __restrict__ occ64, int32_t catalogue,
                                                              int32_t words) {
    const OccBuildGroup& grp = groups[blockIdx.y];
    const uint8_t* sm = slotmask + (size_t)blockIdx.y * np;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool nz = false;
    unsigned long long mk = 0;  // the largest entry this thread writes (its key: entries are >= 0)
    if (i < catalogue) {
        double x[LP];
#pragma unroll
        for (int s = 0; s < LP; ++s) x[s] = 0.0;
        const uint32_t k1 = ptr[i + 1];
        for (uint32_t k = ptr[i]; k < k1; ++k) {
            const SparseEntry en = entries[k];
            const uint32_t mask = sm[en.elt];
            if (!mask) continue;
            const double f = fin_f64((double)en.loss, terms64[en.elt], terms64[np + en.elt], terms64[2 * np + en.elt]);
#pragma unroll
            for (int s = 0; s < LP; ++s)
                if ((mask >> s) & 1u) x[s] += f;
        }
        double o[LP];
#pragma unroll
        for (int s = 0; s < LP; ++s) {
            o[s] = 0.0;
            if (s < grp.n_layers) {
                const int32_t j = grp.layer[s];
                o[s] = xl_f64(x[s], (double)occ_terms[2 * j], (double)occ_terms[2 * j + 1]);
                nz |= o[s] > 0.0;
            }
        }
        double* dst = occ64[blockIdx.y] + i * LP;
        if constexpr (LP == 1) dst[0] = o[0];
        else {
#pragma unroll
            for (int q = 0; q < LP / 2; ++q) reinterpret_cast<double2*>(dst)[q] = make_double2(o[2 * q], o[2 * q + 1]);
        }
#pragma unroll
        for (int s = 0; s < LP; ++s) mk = max(mk, (unsigned long long)__double_as_longlong(o[s]));
    }
    note_max(grp.maxkey, mk);
    const unsigned m = __ballot_sync(0xffffffffu, nz);
    if ((threadIdx.x & 31) == 0 && (i >> 5) < words) grp.occ_bits[i >> 5] = m;
}

// Packs every entry of group blockIdx.y's table in place (fix_pack against
// the group's reference exponent, known once the build has recorded the
// table's largest entry), so that the trial passes add each entry without
// splitting it into mantissa and shift again.
__global__ void __launch_bounds__(256) pack_occ64_kernel(double* const* __restrict__ occ64,
                                                         const OccBuildGroup* __restrict__ groups, int64_t n_entries) {
    const int e_ref = ref_exp(__ldcg(groups[blockIdx.y].maxkey));
    unsigned long long* t = reinterpret_cast<unsigned long long*>(occ64[blockIdx.y]);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_entries;
         i += (int64_t)gridDim.x * blockDim.x)
        t[i] = fix_pack(t[i], e_ref);
}

template <int LT, bool VEC, bool FOLD>
__global__ void __launch_bounds__(k64Threads, 1) ylt_skip64_kernel(const OccGroupArgs g, const YetArgs y,
                                                                  const int32_t smem_words, const bool early_exit,
                                                                  double* __restrict__ ylt,
                                                                  uint8_t* __restrict__ branch,
                                                                  int* __restrict__ flags) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int E = k64Ids;
    extern __shared__ __align__(16) uint32_t s_dyn[];
    int32_t* s_queue = reinterpret_cast<int32_t*>(s_dyn);  // [k64Warps][k64Queue]
    uint32_t* s_bits = s_dyn + k64Warps * k64Queue;
    {
        const uint4* src = reinterpret_cast<const uint4*>(g.occ_bits);
        uint4* dst = reinterpret_cast<uint4*>(s_bits);
        const int words = (y.catalogue >> 5) + 1;  // bits 0 .. C (C: the sentinel)
        for (int i = threadIdx.x; i < smem_words / 4; i += blockDim.x) {
            uint4 v = src[i];
            if (FOLD && 4 * i + smem_words < words) {  // the bitmap is zero-padded to whole uint4
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
    int32_t* q = s_queue + wib * k64Queue;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n_warps = (int64_t)gridDim.x * k64Warps;
    uint32_t max_id = 0;  // largest id seen (an id >= C raises the range flag)
    bool bad_off_seen = false;
    int32_t my_layer = 0;
    double my_ret = 0.0, my_lim = 0.0;
#pragma unroll
    for (int j = 0; j < LT; ++j)
        if (lane == j) {
            my_layer = g.layer[j];
            my_ret = g.agg_ret[j];
            my_lim = g.agg_lim[j];
        }

    // the fixed-point unit: 2^-96 of the group table's largest entry
    const int e_ref = ref_exp(__ldcg(g.maxkey));
    for (int64_t t = (int64_t)blockIdx.x * k64Warps + wib; t < y.n_trials; t += n_warps) {
        int64_t b, e;
        bool bo;
        trial_range(y, t, b, e, bo);
        bad_off_seen |= bo;
        Fix acc[LT];  // the lane's exact per-layer sums
#pragma unroll
        for (int j = 0; j < LT; ++j) acc[j] = Fix{0, 0};
        auto add_row = [&](uint32_t id) {
            unsigned long long o[LT];  // the row's packed entries
            ld_row64<LT>(g.occ64, id, o);
#pragma unroll
            for (int j = 0; j < LT; ++j) fix_add_packed(acc[j], o[j]);
        };
        // ids of a chunk of 32 * E events from c0; empty slots read as -1
        auto load_ids = [&](int64_t c0, uint32_t (&v)[E]) {
            if constexpr (VEC) {
#pragma unroll
                for (int h = 0; h < E / 4; ++h) {
                    const int64_t d = c0 + 128 * h + 4 * lane;
                    int4 w4 = make_int4(-1, -1, -1, -1);
                    if (d < e) w4 = __ldcs(reinterpret_cast<const int4*>(y.ids + d));  // e and d are multiples of 4
                    v[4 * h + 0] = (uint32_t)w4.x;
                    v[4 * h + 1] = (uint32_t)w4.y;
                    v[4 * h + 2] = (uint32_t)w4.z;
                    v[4 * h + 3] = (uint32_t)w4.w;
                }
            } else {
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    const int64_t d = c0 + 32 * k + lane;
                    v[k] = d < e ? (uint32_t)ld_stream(y.ids + d) : 0xffffffffu;
                }
            }
        };
        int qn = 0;  // warp-uniform, < 32 between chunks
        bool capped_exit = false;
        uint32_t pre[E];
        if (b < e) load_ids(b, pre);
        for (int64_t c0 = b; c0 < e; c0 += 32 * E) {
            uint32_t uid[E];
#pragma unroll
            for (int k = 0; k < E; ++k) {
                // slot k's position in the trial (empty slots hold -1: no flag)
                const int64_t d = VEC ? c0 + 128 * (k >> 2) + 4 * lane + (k & 3) : c0 + 32 * k + lane;
                if (d < e) max_id = max(max_id, pre[k]);
                uid[k] = min(pre[k], (uint32_t)y.catalogue);
            }
            if (c0 + 32 * E < e) load_ids(c0 + 32 * E, pre);
#pragma unroll
            for (int k = 0; k < E; ++k) {
                uint32_t wi = uid[k] >> 5;
                uint32_t w;
                if constexpr (FOLD) {
                    wi = min(wi, wi - (uint32_t)smem_words);  // wi - S wraps when wi < S
                    w = s_bits[wi];
                } else {
                    w = wi < (uint32_t)smem_words ? s_bits[wi] : ld_bits_global(g.occ_bits + wi);
                }
                const bool nz = (w >> (uid[k] & 31)) & 1u;
                const unsigned mm = __ballot_sync(FULL, nz);
                if (nz) q[qn + __popc(mm & lt_mask)] = (int32_t)uid[k];
                qn += __popc(mm);
                if (qn >= 32) {
                    __syncwarp();
                    const int32_t mine = q[lane];
                    const int32_t carry = q[32 + lane];
                    __syncwarp();
                    q[lane] = carry;  // entries 32 .. qn-1 move to the front
                    qn -= 32;
                    add_row((uint32_t)mine);
                    __syncwarp();
                }
            }
            if (early_exit) {
                // every layer capped: the aggregate never decreases, the loss is AggL
                bool all = true;
#pragma unroll
                for (int j = 0; j < LT; ++j) {
                    const double v = fix_value(fix_warp_sum(acc[j]), e_ref);
                    if (j < g.n_layers) all = all && (v - g.agg_ret[j] >= g.agg_lim[j]);
                }
                if (all) {
                    qn = 0;
                    capped_exit = true;
                    break;
                }
            }
        }
        __syncwarp();
        if (lane < qn) add_row((uint32_t)q[lane]);
        __syncwarp();
        // lane j keeps layer j's total and converts it: one FP64 conversion
        // per lane rather than one per layer under a one-lane predicate
        Fix mine_f{0, 0};
#pragma unroll
        for (int j = 0; j < LT; ++j) {
            const Fix tot = fix_warp_sum(acc[j]);
            if (lane == j) mine_f = tot;
        }
        const double mine = fix_value(mine_f, e_ref);
        if (lane < g.n_layers) {
            const size_t wi = (size_t)my_layer * (size_t)y.n_trials + (size_t)t;
            ylt[wi] = capped_exit ? my_lim : xl_f64(mine, my_ret, my_lim);
            if (branch) branch[wi] = capped_exit ? (uint8_t)2 : agg_branch(mine, my_ret, my_lim);
        }
    }
    if (max_id >= (uint32_t)y.catalogue) atomicOr(flags + kFlagIdRange, 1);
    if (lane == 0 && bad_off_seen) atomicOr(flags + kFlagBadOffsets, 1);
}

template <int LT>
cudaError_t launch_group64(const OccGroupArgs& g, const YetArgs& y, int num_sms, int32_t catalogue, bool early,
                           double* ylt, uint8_t* branch, int* flags, cudaStream_t s) {
    int dev = 0, max_optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
    const int queue_bytes = k64Warps * k64Queue * 4;
    const int words = (catalogue >> 5) + 1;  // bits 0 .. C (C: the sentinel)
    const int smem_words = std::max(4, std::min((words + 3) & ~3, (max_optin - queue_bytes) / 4) & ~3);
    const int smem = queue_bytes + smem_words * 4;
    const bool fold = words <= 2 * smem_words;
    const bool vec = !y.off && y.k % 4 == 0 && (reinterpret_cast<uintptr_t>(y.ids) & 15) == 0;
    auto kern = vec ? (fold ? ylt_skip64_kernel<LT, true, true> : ylt_skip64_kernel<LT, true, false>)
                    : (fold ? ylt_skip64_kernel<LT, false, true> : ylt_skip64_kernel<LT, false, false>);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    const int64_t grid = std::min<int64_t>(num_sms, (y.n_trials + k64Warps - 1) / k64Warps);
    kern<<<(unsigned)std::max<int64_t>(1, grid), k64Threads, smem, s>>>(g, y, smem_words, early, ylt, branch, flags);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_skip64(art_portfolio* p, const YetArgs& y, double* ylt, uint8_t* branch, cudaStream_t s,
                          bool build) {
    const bool early = (p->flags & ART_FLAG_EARLY_EXIT) != 0;
    const int32_t words = (int32_t)(((int64_t)p->catalogue + 31) / 32);
    const dim3 grid((unsigned)(((int64_t)words * 32 + 255) / 256), (unsigned)p->ogroups64.size());
    // from the CSR of the non-zero losses where it exists, else from the
    // per-layer tables
    const bool csr = p->sp_ptr && p->d_slotmask64 && p->d_elt_terms64 && p->d_occ;
    const SparseEntry* en = reinterpret_cast<const SparseEntry*>(p->sp_entries);
    if (build) {
        cudaError_t me = cudaMemsetAsync(p->d_occ64_max, 0, sizeof(unsigned long long) * p->ogroups64.size(), s);
        if (me != cudaSuccess) return me;
        if (csr) {
            switch (p->og_lp64) {
                case 1: build_occ64_csr_kernel<1><<<grid, 256, 0, s>>>(p->sp_ptr, en, p->d_elt_terms64, p->pool_np, p->d_slotmask64, p->d_occ, p->d_ogroups64, p->d_occ64_ptrs, p->catalogue, words); break;
                case 2: build_occ64_csr_kernel<2><<<grid, 256, 0, s>>>(p->sp_ptr, en, p->d_elt_terms64, p->pool_np, p->d_slotmask64, p->d_occ, p->d_ogroups64, p->d_occ64_ptrs, p->catalogue, words); break;
                case 4: build_occ64_csr_kernel<4><<<grid, 256, 0, s>>>(p->sp_ptr, en, p->d_elt_terms64, p->pool_np, p->d_slotmask64, p->d_occ, p->d_ogroups64, p->d_occ64_ptrs, p->catalogue, words); break;
                default: return cudaErrorInvalidValue;
            }
        } else {
            switch (p->og_lp64) {
                case 1: build_occ64_kernel<1><<<grid, 256, 0, s>>>(p->d_lbuild, p->d_ogroups64, p->d_occ64_ptrs, p->catalogue, words); break;
                case 2: build_occ64_kernel<2><<<grid, 256, 0, s>>>(p->d_lbuild, p->d_ogroups64, p->d_occ64_ptrs, p->catalogue, words); break;
                case 4: build_occ64_kernel<4><<<grid, 256, 0, s>>>(p->d_lbuild, p->d_ogroups64, p->d_occ64_ptrs, p->catalogue, words); break;
                default: return cudaErrorInvalidValue;
            }
        }
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    if (build) {
        // the tables' entries packed against their groups' largest entries
        const int64_t n_entries = ((int64_t)p->catalogue + 1) * p->og_lp64;
        const int64_t blocks = std::min<int64_t>((n_entries + 255) / 256, (int64_t)p->num_sms * 8);
        pack_occ64_kernel<<<dim3((unsigned)blocks, (unsigned)p->ogroups64.size()), 256, 0, s>>>(
            p->d_occ64_ptrs, p->d_ogroups64, n_entries);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    if (y.n_trials == 0) return cudaSuccess;
    for (const OccGroupArgs& g : p->ogroups64) {
        switch (p->og_lp64) {
            case 1: err = launch_group64<1>(g, y, p->num_sms, p->catalogue, early, ylt, branch, p->d_flags, s); break;
            case 2: err = launch_group64<2>(g, y, p->num_sms, p->catalogue, early, ylt, branch, p->d_flags, s); break;
            case 4: err = launch_group64<4>(g, y, p->num_sms, p->catalogue, early, ylt, branch, p->d_flags, s); break;
            default: err = cudaErrorInvalidValue;
        }
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace art

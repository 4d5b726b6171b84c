// adjoint_group.cu -- the adjoint of the forward pass (the pricing
// sensitivity added around Section II's Algorithm 1) over layer groups (up
// to 8 layers whose ELTs number at most 32 together, ART_LAYOUT_GROUP).
//
// With a_j = [branch_j == mid] and c_j = [branch_j == capped] from the
// forward's aggregate branch codes and g_j the trial's weight:
//   dAggR_j = -g_j a_j,  dAggL_j = g_j c_j,
//   dOccR_j = -g_j a_j #{d : OccR_j < x_dj < OccR_j + OccL_j},
//   dOccL_j =  g_j a_j #{d : x_dj > OccR_j + OccL_j},
//   dm_e    = sum_d [D_e < m_e l_de < D_e + Lim_e] l_de w_de,
//             w_de = sum_{j covering e} g_j a_j [o_dj on its middle branch].
//
// Which occurrence branch each layer takes, and which ELT terms are on their
// middle branch, depend on the event id alone. So each call first evaluates
// them once per catalogue event i (the group table row, F_e and the layer
// sums x_ij in FP32, in the group's ELT order): M_i, the layers on the middle
// branch; K_i, the layers on the capped branch; and U_i, the ELT columns on
// their middle branch; plus a bitmap of the events with M_i or K_i non-zero
// (only those contribute). The trial pass is then shaped like the forward's:
// a persistent CTA per SM with the bitmap in shared memory (folded once when
// it does not fit), a warp per trial streaming its ids, and a per-warp queue
// of the events whose bit is set, evaluated 32 at a time (lane = event):
//   - the layer counts: per lane, 8-bit counters for the 8 layers packed in
//     a 64-bit word, incremented by a table lookup of M (and K); reduced
//     across the warp with integer reductions at the end of the trial (and
//     every 255 batches), then lane j adds layer j's counts times g_j (g_j
//     rounded to FP32, the product exact) to a compensated FP32 pair;
//   - the multipliers: for each column k in U_i with M_i non-zero, the lane
//     adds l_ik * W[M_i & C_k] to its FP32 partial of column k, where C_k is
//     the set of layers covering column k and W[S] = sum_{j in S} g_j a_j is
//     a 2^LT-entry table of the trial's weights (FP32, per warp, built per
//     trial); at the end of the trial the partials are summed across the
//     warp (recursive halving: 31 shuffles for every column at once) and
//     lane k adds column k's total to its compensated FP32 pair.
// A trial with no layer on the middle branch costs only its branch codes.
// The lane values are reduced warp -> CTA -> grid in a fixed order (no
// atomics: deterministic); FP64 arithmetic runs only in that final
// reduction. Rounding: g is rounded to FP32 once per (layer, trial), and the
// per-event products and the W entries are FP32 (a few units in the last
// place of FP32 per term); every sum is compensated or FP64.
#include <algorithm>
#include <limits>

#include "art_internal.cuh"

namespace art {

namespace {

// Threads per CTA of the trial pass and ids per lane in flight, by the
// group's column count. Up to 16 columns the pass needs about 80 registers
// per thread, and 24 warps per SM with 4 ids each hide more of the gathers'
// latency than 16 warps with 8 ids (c3 adjoint 3.88 against 4.18 ms; 1024
// threads spill); wider groups keep 512 threads with 8 ids (128 registers,
// no spills).
template <int NP>
constexpr int kAgThreadsFor = NP <= 16 ? 768 : 512;
template <int NP>
constexpr int kAgIdsFor = NP <= 16 ? 4 : 8;
constexpr int kAgQueue = 64;  // per-warp queue entries

__device__ __forceinline__ uint32_t ld_bits_global(const uint32_t* p) {
    uint32_t v;
    asm("ld.global.nc.L1::evict_last.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ uint2 ld_mask(const uint2* p) {
    uint2 v;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
    return v;
}

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

// (h, l) += v, keeping the rounding error of the FP32 add (two-sum)
__device__ __forceinline__ void two_sum_add(float& h, float& l, float v) {
    const float t = h + v;
    const float bp = t - h;
    l += (h - (t - bp)) + (v - bp);
    h = t;
}

// Per catalogue event i of a group: masks[i] = (M | K << 8, U) and bit i of
// the bitmap set when M | K is non-zero. Row C (the sentinel for ids outside
// the catalogue) is never written: it stays zero.
template <int NP, int LT>
__global__ void __launch_bounds__(256) adj_masks_kernel(const GroupArgs g, int32_t catalogue, int32_t words,
                                                        uint2* __restrict__ masks, uint32_t* __restrict__ bits) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool rel = false;
    if (i < catalogue) {
        const float4* row = reinterpret_cast<const float4*>(g.table) + i * (NP / 4);
        float v[NP];
#pragma unroll
        for (int q = 0; q < NP / 4; ++q) {
            const float4 r = __ldcs(row + q);
            v[4 * q + 0] = r.x;
            v[4 * q + 1] = r.y;
            v[4 * q + 2] = r.z;
            v[4 * q + 3] = r.w;
        }
        float f[NP];
        uint32_t u = 0u;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            const float wf = __fmaf_rn(g.m[k], v[k], -g.d[k]);
            f[k] = fminf(fmaxf(wf, 0.0f), g.lim[k]);
            if (wf > 0.0f && wf < g.lim[k]) u |= 1u << k;
        }
        uint32_t mk = 0u;
#pragma unroll
        for (int j = 0; j < LT; ++j) {
            if (j < g.n_layers) {
                float x = 0.0f;
#pragma unroll
                for (int k = 0; k < NP; ++k) {
                    if constexpr (LT == 1) x += f[k];
                    else x = __fmaf_rn(g.coef[j][k], f[k], x);
                }
                const float wo = x - g.occ_ret[j];  // the forward's occurrence subtraction
                if (wo > 0.0f && wo < g.occ_lim[j]) mk |= 1u << j;
                if (wo > g.occ_lim[j]) mk |= 1u << (8 + j);
            }
        }
        masks[i] = make_uint2(mk, (mk & 0xffu) ? u : 0u);
        rel = mk != 0u;
    }
    const unsigned m = __ballot_sync(0xffffffffu, rel);
    if ((threadIdx.x & 31) == 0 && (i >> 5) < words) bits[i >> 5] = m;
}

// One queued event on one lane: the packed layer counters and, when a layer
// is on its middle branch, the column partials.
template <int NP, int LT>
__device__ __forceinline__ void eval_event(const GroupArgs& g, const uint2* __restrict__ masks, uint32_t id,
                                           uint32_t last_row, const uint64_t* s_spread, const float* s_w, const uint32_t* s_col,
                                           uint64_t& cnt_mid, uint64_t& cnt_cap, float (&part)[NP]) {
    // the row is requested together with the masks (most queued events need
    // it), so the two gathers overlap; the sentinel C (zero masks) reads the
    // last row instead, unused
    const uint2 mk = ld_mask(masks + id);
    const float* row = g.table + (size_t)min(id, last_row) * NP;
    float v[NP];
    if constexpr (NP % 8 == 0) {
#pragma unroll
        for (int q = 0; q < NP / 8; ++q) ld_row8(row + 8 * q, v + 8 * q);
    } else {
#pragma unroll
        for (int q = 0; q < NP / 4; ++q) ld_row4(row + 4 * q, v + 4 * q);
    }
    const uint32_t m = mk.x & 0xffu;
    cnt_mid += s_spread[m];
    cnt_cap += s_spread[(mk.x >> 8) & 0xffu];
    if (mk.y != 0u) {  // U is stored only where M is non-zero
#pragma unroll
        for (int k = 0; k < NP; ++k)
            if ((mk.y >> k) & 1u) part[k] = __fmaf_rn(v[k], s_w[m & s_col[k]], part[k]);
    }
}

template <int NP, int LT, bool VEC, bool FOLD>
__global__ void __launch_bounds__(kAgThreadsFor<NP>, 1) adjoint_pass_kernel(const GroupArgs g, const YetArgs y,
                                                                     const uint2* __restrict__ masks,
                                                                     const uint32_t* __restrict__ gbits,
                                                                     const int32_t smem_words,
                                                                     const uint8_t* __restrict__ branch,
                                                                     const double* __restrict__ gw,
                                                                     double* __restrict__ partial) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int E = kAgIdsFor<NP>;
    constexpr int kAgWarps = kAgThreadsFor<NP> / 32;
    constexpr int NW = 1 << LT;      // entries of a warp's weight table
    constexpr int W = 4 * LT + NP;   // OccR[LT], OccL[LT], AggR[LT], AggL[LT], then the columns
    extern __shared__ __align__(16) uint32_t s_dyn[];
    uint64_t* s_spread = reinterpret_cast<uint64_t*>(s_dyn);            // [256]
    double* s_red = reinterpret_cast<double*>(s_dyn + 512);              // [kAgWarps][W]
    uint32_t* s_col = s_dyn + 512 + 2 * kAgWarps * W;                    // [32]
    float* s_wt = reinterpret_cast<float*>(s_col + 32);                  // [kAgWarps][NW]
    int32_t* s_queue = reinterpret_cast<int32_t*>(s_wt + kAgWarps * NW); // [kAgWarps][kAgQueue]
    uint32_t* s_bits = reinterpret_cast<uint32_t*>(s_queue + kAgWarps * kAgQueue);
    {
        // s_spread[m]: byte j is bit j of m (adds one to layer j's counter)
        for (int m = threadIdx.x; m < 256; m += blockDim.x) {
            uint64_t v = 0;
            for (int j = 0; j < 8; ++j) v |= (uint64_t)((m >> j) & 1) << (8 * j);
            s_spread[m] = v;
        }
        if (threadIdx.x < 32) {
            uint32_t c = 0;
            for (int j = 0; j < LT; ++j)
                if (j < g.n_layers) c |= ((g.member[j] >> threadIdx.x) & 1u) << j;
            s_col[threadIdx.x] = c;
        }
        const uint4* src = reinterpret_cast<const uint4*>(gbits);
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
    int32_t* q = s_queue + wib * kAgQueue;
    float* s_w = s_wt + wib * NW;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n_warps = (int64_t)gridDim.x * kAgWarps;

    // lane j < LT keeps layer j's four term sums, lane k < NP column k's sum,
    // each a compensated FP32 pair (FP64 arithmetic per trial would dominate:
    // the FP64 pipe of this part is slow)
    float or_h = 0.0f, or_l = 0.0f, ol_h = 0.0f, ol_l = 0.0f, ar_h = 0.0f, ar_l = 0.0f, al_h = 0.0f, al_l = 0.0f;
    float col_h = 0.0f, col_l = 0.0f;
    int32_t my_layer = -1;
#pragma unroll
    for (int j = 0; j < LT; ++j)
        if (lane == j && j < g.n_layers) my_layer = g.layer[j];

    for (int64_t t = (int64_t)blockIdx.x * kAgWarps + wib; t < y.n_trials; t += n_warps) {
        float gt = 0.0f;  // the layer's weight, rounded to FP32 once
        uint8_t code = 0;
        if (my_layer >= 0) {
            const size_t wi = (size_t)my_layer * (size_t)y.n_trials + (size_t)t;
            code = branch[wi];
            gt = (float)gw[wi];
        }
        if (code == 1) two_sum_add(ar_h, ar_l, -gt);
        if (code == 2) two_sum_add(al_h, al_l, gt);
        const bool mid_l = code == 1 && gt != 0.0f;
        if (!__ballot_sync(FULL, mid_l)) continue;  // no layer of the group has a middle-branch weight
        // the trial's weight table W[S] = sum_{j in S} g_j a_j, by doubling:
        // W[S + 2^b] = W[S] + g_b a_b for S < 2^b (the terms in increasing j,
        // as a direct sum adds them)
        {
            if (lane == 0) s_w[0] = 0.0f;
            __syncwarp();
#pragma unroll
            for (int b = 0; b < LT; ++b) {
                const float gb = __shfl_sync(FULL, mid_l ? gt : 0.0f, b);
                for (int s = lane; s < (1 << b); s += 32) s_w[s + (1 << b)] = s_w[s] + gb;
                __syncwarp();
            }
        }
        uint64_t cnt_mid = 0, cnt_cap = 0;
        float part[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) part[k] = 0.0f;
        // lane j adds the warp's counts of layer j, scaled by g_j, and clears
        // them; the products are exact (FMA residual), the sums compensated
        auto flush_counts = [&]() {
#pragma unroll
            for (int j = 0; j < LT; ++j) {
                const uint32_t cm = __reduce_add_sync(FULL, (uint32_t)(cnt_mid >> (8 * j)) & 0xffu);
                const uint32_t cc = __reduce_add_sync(FULL, (uint32_t)(cnt_cap >> (8 * j)) & 0xffu);
                if (lane == j && mid_l) {
                    const float pm = gt * (float)cm, pc = gt * (float)cc;  // counts < 2^24: exact in FP32
                    two_sum_add(or_h, or_l, -pm);
                    or_l -= __fmaf_rn(gt, (float)cm, -pm);
                    two_sum_add(ol_h, ol_l, pc);
                    ol_l += __fmaf_rn(gt, (float)cc, -pc);
                }
            }
            cnt_mid = 0;
            cnt_cap = 0;
        };
        int64_t b, e;
        bool bad_off;
        trial_range(y, t, b, e, bad_off);
        int qn = 0;        // warp-uniform, < 32 between chunks
        int batches = 0;   // batches since the counters were cleared (each lane's byte counters < 256)
        // ids of a chunk of 32 * E events from c0 (the sentinel C past the end)
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
        uint32_t pre[E];
        if (b < e) load_ids(b, pre);
        for (int64_t c0 = b; c0 < e; c0 += 32 * E) {
            uint32_t uid[E];
#pragma unroll
            for (int k = 0; k < E; ++k) uid[k] = min(pre[k], (uint32_t)y.catalogue);
            // request the trial's next chunk before this one is processed
            if (c0 + 32 * E < e) load_ids(c0 + 32 * E, pre);
#pragma unroll
            for (int k = 0; k < E; ++k) {
                uint32_t wi = uid[k] >> 5;
                uint32_t w;
                if constexpr (FOLD) {
                    wi = wi >= (uint32_t)smem_words ? wi - (uint32_t)smem_words : wi;
                    w = s_bits[wi];
                } else {
                    w = wi < (uint32_t)smem_words ? s_bits[wi] : ld_bits_global(gbits + wi);
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
                    eval_event<NP, LT>(g, masks, (uint32_t)mine, (uint32_t)y.catalogue - 1u, s_spread, s_w, s_col, cnt_mid, cnt_cap, part);
                    if (++batches == 255) {
                        flush_counts();
                        batches = 0;
                    }
                    __syncwarp();
                }
            }
        }
        __syncwarp();
        if (lane < qn) eval_event<NP, LT>(g, masks, (uint32_t)q[lane], (uint32_t)y.catalogue - 1u, s_spread, s_w, s_col, cnt_mid, cnt_cap, part);
        __syncwarp();
        flush_counts();
        // the trial's column partials summed across the warp by recursive
        // halving (31 shuffles for all columns): at distance o a lane keeps
        // the half of its columns selected by bit o of its index and adds
        // the partner's copy of that half; lane k ends with column k
        {
            float v[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) v[k] = k < NP ? part[k] : 0.0f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const bool upper = (lane & o) != 0;
#pragma unroll
                for (int i = 0; i < o; ++i) {
                    const float keep = upper ? v[i + o] : v[i];
                    const float send = upper ? v[i] : v[i + o];
                    v[i] = keep + __shfl_xor_sync(FULL, send, o);
                }
            }
            if (lane < NP) two_sum_add(col_h, col_l, v[0]);
        }
        __syncwarp();  // the weight table is rebuilt by the next trial
    }
    // the lane values in FP64, reduced warp -> CTA in a fixed order
#pragma unroll
    for (int i = 0; i < W; ++i) {
        double v;
        if (i < 4 * LT) {
            const int c = i / LT, j = i % LT;
            const double mine = c == 0   ? (double)or_h + (double)or_l
                                : c == 1 ? (double)ol_h + (double)ol_l
                                : c == 2 ? (double)ar_h + (double)ar_l
                                         : (double)al_h + (double)al_l;
            v = lane == j ? mine : 0.0;
        } else {
            v = lane == i - 4 * LT ? (double)col_h + (double)col_l : 0.0;
        }
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
        if (lane == 0) s_red[wib * W + i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        double s = 0.0;
        for (int wv = 0; wv < kAgWarps; ++wv) s += s_red[wv * W + i];
        partial[(size_t)blockIdx.x * W + i] = s;
    }
}

// The group's ELT ids (union order) and layer ids, passed by value.
struct GroupIndex {
    int32_t elt[kMaxLayerElts];
    int32_t layer[kMaxGroupLayers];
    int32_t n_elt, n_layers;
};

// Sum the CTA partials of one group in block order and add them into the
// outputs: each layer belongs to one group; an ELT's multiplier gradient sums
// over the groups that hold it, in group order (groups run in order on one
// stream).
__global__ void group_scatter_kernel(const double* __restrict__ partial, int nblk, int lt, int np,
                                     const GroupIndex gix, double* __restrict__ grad_terms,
                                     double* __restrict__ grad_mult) {
    const int w = 4 * lt + np;
    const int i = threadIdx.x;
    if (i >= w) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * w + i];
    if (i < 4 * lt) {
        const int c = i / lt, j = i % lt;
        if (j < gix.n_layers) grad_terms[(size_t)gix.layer[j] * 4 + c] = s;
    } else {
        const int k = i - 4 * lt;
        if (k < gix.n_elt) grad_mult[gix.elt[k]] += s;
    }
}

struct Scratch {
    uint2* masks;     // [C + 1]
    uint32_t* bits;   // zero-padded to whole 16-byte groups, bits 0 .. C
    double* partial;  // [num_sms][4 * 8 + 32]
};

template <int NP, int LT>
cudaError_t launch_one(const GroupArgs& g, const GroupIndex& gix, const YetArgs& y, const uint8_t* branch,
                       const double* gw, const Scratch& sc, int num_sms, double* grad_terms, double* grad_mult,
                       cudaStream_t s) {
    const int32_t C = y.catalogue;
    const int32_t words_w = (int32_t)(((int64_t)C + 31) / 32);  // words the mask kernel writes
    adj_masks_kernel<NP, LT><<<(unsigned)(((int64_t)words_w * 32 + 255) / 256), 256, 0, s>>>(g, C, words_w, sc.masks,
                                                                                            sc.bits);
    cudaError_t e = cudaGetLastError();
    if (e || y.n_trials == 0) return e;
    int dev = 0, max_optin = 0;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev))) return e;
    constexpr int W = 4 * LT + NP;
    constexpr int kAgWarps = kAgThreadsFor<NP> / 32;
    const int fixed = 4 * (512 + 2 * kAgWarps * W + 32 + kAgWarps * (1 << LT) + kAgWarps * kAgQueue);
    const int words = (C >> 5) + 1;  // bits 0 .. C (C: the sentinel)
    const int smem_words = std::max(4, std::min((words + 3) & ~3, (max_optin - fixed) / 4) & ~3);
    const int smem = fixed + 4 * smem_words;
    const bool fold = words <= 2 * smem_words;
    const bool vec = !y.off && y.k % 4 == 0 && (reinterpret_cast<uintptr_t>(y.ids) & 15) == 0;
    auto kern = vec ? (fold ? adjoint_pass_kernel<NP, LT, true, true> : adjoint_pass_kernel<NP, LT, true, false>)
                    : (fold ? adjoint_pass_kernel<NP, LT, false, true> : adjoint_pass_kernel<NP, LT, false, false>);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(num_sms, (y.n_trials + kAgWarps - 1) / kAgWarps));
    kern<<<nblk, kAgThreadsFor<NP>, smem, s>>>(g, y, sc.masks, sc.bits, smem_words, branch, gw, sc.partial);
    if ((e = cudaGetLastError())) return e;
    group_scatter_kernel<<<1, 128, 0, s>>>(sc.partial, nblk, LT, NP, gix, grad_terms, grad_mult);
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch_lt(const GroupArgs& g, const GroupIndex& gix, const YetArgs& y, const uint8_t* branch,
                      const double* gw, const Scratch& sc, int num_sms, double* gt, double* gm, cudaStream_t s) {
    if (g.n_layers <= 1) return launch_one<NP, 1>(g, gix, y, branch, gw, sc, num_sms, gt, gm, s);
    if (g.n_layers <= 2) return launch_one<NP, 2>(g, gix, y, branch, gw, sc, num_sms, gt, gm, s);
    if (g.n_layers <= 4) return launch_one<NP, 4>(g, gix, y, branch, gw, sc, num_sms, gt, gm, s);
    return launch_one<NP, 8>(g, gix, y, branch, gw, sc, num_sms, gt, gm, s);
}

}  // namespace

cudaError_t launch_adjoint_groups(art_portfolio* p, const YetArgs& y, const uint8_t* branch, const double* g,
                                  double* grad_terms, double* grad_mult, cudaStream_t s) {
    const size_t C = (size_t)p->catalogue;
    const size_t mask_bytes = sizeof(uint2) * (C + 1);
    const size_t bit_bytes = 16 * ((C / 32 + 1 + 3) / 4);
    const size_t part_bytes = sizeof(double) * (size_t)p->num_sms * (4 * kMaxGroupLayers + kMaxLayerElts);
    const size_t a1 = (mask_bytes + 255) & ~(size_t)255, a2 = (bit_bytes + 255) & ~(size_t)255;
    char* w = nullptr;
    cudaError_t err = cudaMallocAsync((void**)&w, a1 + a2 + part_bytes, s);
    if (err) return err;
    Scratch sc{reinterpret_cast<uint2*>(w), reinterpret_cast<uint32_t*>(w + a1), reinterpret_cast<double*>(w + a1 + a2)};
    do {
        if ((err = cudaMemsetAsync(grad_terms, 0, sizeof(double) * 4 * p->n_layers, s))) break;
        if ((err = cudaMemsetAsync(grad_mult, 0, sizeof(double) * p->n_elt, s))) break;
        if (y.n_trials == 0) break;
        // the sentinel row and the padding words stay zero for every group
        if ((err = cudaMemsetAsync(w, 0, a1 + a2, s))) break;
        for (size_t gi = 0; gi < p->groups.size() && !err; ++gi) {
            const GroupArgs& ga = p->groups[gi];
            GroupIndex gix{};
            gix.n_elt = (int32_t)p->group_elts[gi].size();
            gix.n_layers = (int32_t)p->group_layers[gi].size();
            for (int k = 0; k < gix.n_elt; ++k) gix.elt[k] = p->group_elts[gi][k];
            for (int j = 0; j < gix.n_layers; ++j) gix.layer[j] = p->group_layers[gi][j];
            const int ns = p->num_sms;
            double* gt = grad_terms;
            double* gm = grad_mult;
            switch (p->group_np[gi]) {
                case 4: err = launch_lt<4>(ga, gix, y, branch, g, sc, ns, gt, gm, s); break;
                case 8: err = launch_lt<8>(ga, gix, y, branch, g, sc, ns, gt, gm, s); break;
                case 16: err = launch_lt<16>(ga, gix, y, branch, g, sc, ns, gt, gm, s); break;
                case 24: err = launch_lt<24>(ga, gix, y, branch, g, sc, ns, gt, gm, s); break;
                case 32: err = launch_lt<32>(ga, gix, y, branch, g, sc, ns, gt, gm, s); break;
                default: err = cudaErrorInvalidValue;
            }
        }
    } while (0);
    const cudaError_t e2 = cudaFreeAsync(w, s);
    return err ? err : e2;
}

}  // namespace art

// adjoint_group.cu -- the adjoint of the forward pass (the pricing
// sensitivity added around Section II's Algorithm 1) over layer groups: one
// pass over the YET per group of up to 8 layers rather than one per layer,
// and only the events whose bit is set in the group's occupancy bitmap are
// evaluated (an event with a clear bit has x_dj = 0 for every layer j of the
// group, which lies on no middle branch, so it contributes nothing).
//
// With a_j = [branch_j == mid] and c_j = [branch_j == capped] from the
// forward's aggregate branch codes and g_j the trial's weight:
//   dAggR_j = -g_j a_j,  dAggL_j = g_j c_j,
//   dOccR_j = -g_j a_j #{d : OccR_j < x_dj < OccR_j + OccL_j},
//   dOccL_j =  g_j a_j #{d : x_dj > OccR_j + OccL_j},
//   dm_e    = sum_d [D_e < m_e l_de < D_e + Lim_e] l_de w_de,
//             w_de = sum_{j covering e} g_j a_j [o_dj on its middle branch].
// The per-event sums x_dj are recomputed in FP32 in the group table's ELT
// order, exactly as the group forward (the skip variant) forms them.
//
// Mapping: warp per trial over a persistent grid (static stride). Lanes
// 0..LT-1 read the trial's branch code and weight of their layer; a trial
// with no layer on the middle branch costs nothing more. Otherwise the warp
// streams the trial's ids 32 * E at a time, tests their bits, queues the
// events with a loss in shared memory and evaluates them 32 at a time (lane =
// event). Per event: the row (one 256-bit load per 8 columns), F_e and its
// middle-branch test per column, the layer sums over their member columns,
// each layer's occurrence branch, the weights w_de (FMA chains with 0/1
// coefficients) and, where non-zero, l_de w_de added to the lane's compensated
// FP32 pair of column e (the lanes' pairs live in shared memory, one column
// per lane, so they cost no registers; few columns of a row are non-zero).
// After each batch the branch flags are counted across the warp (integer
// reductions) on lane j, which scales its layer's counts by g_j in FP64 at
// the end of the trial; so FP64 runs per trial, not per event. The final per-lane
// values are reduced warp -> CTA in a fixed order, and the CTA partials are
// summed in block order (no atomics: deterministic).
#include <algorithm>
#include <limits>

#include "art_internal.cuh"

namespace art {

namespace {

constexpr int kAgThreads = 256;
constexpr int kAgWarps = kAgThreads / 32;
constexpr int kAgIds = 8;                   // ids per lane per chunk
constexpr int kAgQueue = 32 * kAgIds + 32;  // per-warp queue: a chunk plus a partial batch

// hi + lo += v without losing the rounding error of the FP32 add (two-sum)
__device__ __forceinline__ void two_sum_add(float2& a, float v) {
    const float t = a.x + v;
    const float bp = t - a.x;
    a.y += (a.x - (t - bp)) + (v - bp);
    a.x = t;
}

__device__ __forceinline__ uint32_t ld_bits(const uint32_t* p) {
    uint32_t v;
    asm("ld.global.nc.L1::evict_last.u32 %0, [%1];" : "=r"(v) : "l"(p));
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

// One event on one lane. Returns the layers on their middle (bits 0..7) and
// capped (bits 8..15) occurrence branches; adds l w to the lane's pair of
// each column on its middle branch with a non-zero weight. acc is the lane's
// column of pairs in shared memory (stride 32).
template <int NP, int LT>
__device__ __forceinline__ uint32_t eval_adjoint(const GroupArgs& g, int32_t id, const float (&ga)[LT],
                                                 float2* acc) {
    const float* row = g.table + (size_t)id * NP;
    float v[NP];
    if constexpr (NP % 8 == 0) {
#pragma unroll
        for (int q = 0; q < NP / 8; ++q) ld_row8(row + 8 * q, v + 8 * q);
    } else {
#pragma unroll
        for (int q = 0; q < NP / 4; ++q) ld_row4(row + 4 * q, v + 4 * q);
    }
    float f[NP];
    uint32_t fmid = 0u;  // bit k: F_k on its middle branch
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const float wf = __fmaf_rn(g.m[k], v[k], -g.d[k]);
        f[k] = fminf(fmaxf(wf, 0.0f), g.lim[k]);
        if (wf > 0.0f && wf < g.lim[k]) fmid |= 1u << k;
    }
    uint32_t bits = 0u;
    float mw[LT];  // g_j a_j [o_dj on its middle branch]
#pragma unroll
    for (int j = 0; j < LT; ++j) {
        float x = 0.0f;
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            // member columns in the group's ELT order (the same roundings as
            // the forward's 0/1-coefficient FMA chain)
            if (LT == 1 || (g.member[j] & (1u << k))) x += f[k];
        }
        const float wo = x - g.occ_ret[j];  // the forward's occurrence subtraction
        const bool mid = wo > 0.0f && wo < g.occ_lim[j];
        if (mid) bits |= 1u << j;
        if (wo > g.occ_lim[j]) bits |= 1u << (8 + j);
        mw[j] = mid ? ga[j] : 0.0f;
    }
    if (bits & 0xffu) {
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            if ((fmid >> k) & 1u) {
                float wk = 0.0f;
#pragma unroll
                for (int j = 0; j < LT; ++j) {
                    if constexpr (LT == 1) wk += mw[j];
                    else wk = __fmaf_rn(g.coef[j][k], mw[j], wk);
                }
                if (wk != 0.0f) {
                    float2 a = acc[32 * k];
                    two_sum_add(a, v[k] * wk);
                    acc[32 * k] = a;
                }
            }
        }
    }
    return bits;
}

// Lane j < LT adds the warp's count of events on layer j's middle and capped
// occurrence branches.
template <int LT>
__device__ __forceinline__ void count_branches(uint32_t bits, int lane, uint32_t& n_mid, uint32_t& n_cap) {
#pragma unroll
    for (int j = 0; j < LT; ++j) {
        const uint32_t m = __reduce_add_sync(0xffffffffu, (bits >> j) & 1u);
        const uint32_t c = __reduce_add_sync(0xffffffffu, (bits >> (8 + j)) & 1u);
        if (lane == j) {
            n_mid += m;
            n_cap += c;
        }
    }
}

template <int NP, int LT>
__global__ void __launch_bounds__(kAgThreads, 2) adjoint_group_kernel(const GroupArgs g, const YetArgs y,
                                                                      const uint8_t* __restrict__ branch,
                                                                      const double* __restrict__ gw,
                                                                      double* __restrict__ partial) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int E = kAgIds;
    constexpr int W = 4 * LT + NP;  // OccR[LT], OccL[LT], AggR[LT], AggL[LT], then the columns
    extern __shared__ __align__(16) float2 s_acc[];  // [kAgWarps][NP][32]: every lane's column pairs
    __shared__ int32_t s_queue[kAgWarps][kAgQueue];
    __shared__ double s_red[kAgWarps][W];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int32_t* q = s_queue[wib];
    float2* acc = s_acc + (size_t)wib * NP * 32 + lane;
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[32 * k] = make_float2(0.0f, 0.0f);
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n_warps = (int64_t)gridDim.x * kAgWarps;

    // lane j < LT keeps layer j's four term sums
    double acc_or = 0.0, acc_ol = 0.0, acc_ar = 0.0, acc_al = 0.0;
    int32_t my_layer = -1;
#pragma unroll
    for (int j = 0; j < LT; ++j)
        if (lane == j && j < g.n_layers) my_layer = g.layer[j];

    for (int64_t t = (int64_t)blockIdx.x * kAgWarps + wib; t < y.n_trials; t += n_warps) {
        double gt = 0.0;
        uint8_t code = 0;
        if (my_layer >= 0) {
            const size_t wi = (size_t)my_layer * (size_t)y.n_trials + (size_t)t;
            code = branch[wi];
            gt = gw[wi];
        }
        if (code == 1) acc_ar -= gt;
        if (code == 2) acc_al += gt;
        const bool mid_l = code == 1 && gt != 0.0;
        if (!__ballot_sync(FULL, mid_l)) continue;  // no layer of the group has a middle-branch weight
        float ga[LT];
#pragma unroll
        for (int j = 0; j < LT; ++j) ga[j] = __shfl_sync(FULL, mid_l ? (float)gt : 0.0f, j);
        uint32_t n_mid = 0, n_cap = 0;
        int64_t b, e;
        bool bad_off;
        trial_range(y, t, b, e, bad_off);
        int qn = 0;  // warp-uniform, < 32 between chunks
        for (int64_t c0 = b; c0 < e; c0 += 32 * E) {
            int32_t id[E];
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int64_t d = c0 + 32 * k + lane;
                id[k] = d < e ? ld_stream(y.ids + d) : -1;
            }
            uint32_t word[E];
#pragma unroll
            for (int k = 0; k < E; ++k)
                word[k] = (unsigned)id[k] < (unsigned)y.catalogue ? ld_bits(g.bitmap + (id[k] >> 5)) : 0u;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const bool nz = (word[k] >> (id[k] & 31)) & 1u;
                const unsigned m = __ballot_sync(FULL, nz);
                if (nz) q[qn + __popc(m & lt_mask)] = id[k];
                qn += __popc(m);
            }
            // evaluate full batches of 32 from the top of the queue
            while (qn >= 32) {
                __syncwarp();
                const int32_t mine = q[qn - 32 + lane];
                __syncwarp();
                qn -= 32;
                const uint32_t bits = eval_adjoint<NP, LT>(g, mine, ga, acc);
                count_branches<LT>(bits, lane, n_mid, n_cap);
            }
        }
        __syncwarp();
        if (qn > 0) {
            const int32_t mine = lane < qn ? q[lane] : -1;
            __syncwarp();
            const uint32_t bits = mine >= 0 ? eval_adjoint<NP, LT>(g, mine, ga, acc) : 0u;
            count_branches<LT>(bits, lane, n_mid, n_cap);
        }
        // the trial's occurrence counts, scaled by the layer's weight, on lane j
        if (mid_l) {
            acc_or -= gt * (double)n_mid;
            acc_ol += gt * (double)n_cap;
        }
    }
    // the lane values in FP64, reduced warp -> CTA in a fixed order
#pragma unroll
    for (int i = 0; i < W; ++i) {
        double v;
        if (i < 4 * LT) {
            const int c = i / LT, j = i % LT;
            const double mine = c == 0 ? acc_or : c == 1 ? acc_ol : c == 2 ? acc_ar : acc_al;
            v = lane == j ? mine : 0.0;
        } else {
            const float2 a = acc[32 * (i - 4 * LT)];
            v = (double)a.x + (double)a.y;
        }
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
        if (lane == 0) s_red[wib][i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        double s = 0.0;
        for (int wv = 0; wv < kAgWarps; ++wv) s += s_red[wv][i];
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

template <int NP, int LT>
cudaError_t launch_one(const GroupArgs& g, const GroupIndex& gix, const YetArgs& y, const uint8_t* branch,
                       const double* gw, double* partial, int num_sms, int max_blocks, double* grad_terms,
                       double* grad_mult, cudaStream_t s) {
    const int smem = (int)sizeof(float2) * kAgWarps * NP * 32;
    auto kern = adjoint_group_kernel<NP, LT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int per_sm = 0;
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kAgThreads, smem);
    if (e) return e;
    const int nblk = std::max(1, std::min(max_blocks, num_sms * std::max(1, per_sm)));
    kern<<<nblk, kAgThreads, smem, s>>>(g, y, branch, gw, partial);
    if ((e = cudaGetLastError())) return e;
    group_scatter_kernel<<<1, 128, 0, s>>>(partial, nblk, LT, NP, gix, grad_terms, grad_mult);
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch_lt(const GroupArgs& g, const GroupIndex& gix, const YetArgs& y, const uint8_t* branch,
                      const double* gw, double* partial, int num_sms, int max_blocks, double* gt, double* gm,
                      cudaStream_t s) {
    if (g.n_layers <= 1) return launch_one<NP, 1>(g, gix, y, branch, gw, partial, num_sms, max_blocks, gt, gm, s);
    if (g.n_layers <= 2) return launch_one<NP, 2>(g, gix, y, branch, gw, partial, num_sms, max_blocks, gt, gm, s);
    if (g.n_layers <= 4) return launch_one<NP, 4>(g, gix, y, branch, gw, partial, num_sms, max_blocks, gt, gm, s);
    return launch_one<NP, 8>(g, gix, y, branch, gw, partial, num_sms, max_blocks, gt, gm, s);
}

}  // namespace

cudaError_t launch_adjoint_groups(art_portfolio* p, const YetArgs& y, const uint8_t* branch, const double* g,
                                  double* grad_terms, double* grad_mult, cudaStream_t s) {
    // at most 8 CTAs of 256 threads are resident per SM
    const int max_blocks = p->num_sms * 8;
    const size_t part_bytes = sizeof(double) * (size_t)max_blocks * (4 * kMaxGroupLayers + kMaxLayerElts);
    double* partial = nullptr;
    cudaError_t err = cudaMallocAsync((void**)&partial, part_bytes, s);
    if (err) return err;
    do {
        if ((err = cudaMemsetAsync(grad_terms, 0, sizeof(double) * 4 * p->n_layers, s))) break;
        if ((err = cudaMemsetAsync(grad_mult, 0, sizeof(double) * p->n_elt, s))) break;
        if (y.n_trials == 0) break;
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
                case 4: err = launch_lt<4>(ga, gix, y, branch, g, partial, ns, max_blocks, gt, gm, s); break;
                case 8: err = launch_lt<8>(ga, gix, y, branch, g, partial, ns, max_blocks, gt, gm, s); break;
                case 16: err = launch_lt<16>(ga, gix, y, branch, g, partial, ns, max_blocks, gt, gm, s); break;
                case 24: err = launch_lt<24>(ga, gix, y, branch, g, partial, ns, max_blocks, gt, gm, s); break;
                case 32: err = launch_lt<32>(ga, gix, y, branch, g, partial, ns, max_blocks, gt, gm, s); break;
                default: err = cudaErrorInvalidValue;
            }
        }
    } while (0);
    const cudaError_t e2 = cudaFreeAsync(partial, s);
    return err ? err : e2;
}

}  // namespace art

// ylt_skip.cu -- the forward pass for layer groups with an occupancy bitmap
// (Section II, Algorithm 1; Section III's direct-access tables, plus the
// occupancy summary that Section VI's compressed representations point to).
//
// A group is up to 8 layers whose ELTs together number at most 32. It has a
// direct-access table [C][np] FP32 over the union of its ELTs (event-major)
// and a bitmap over the catalogue: bit i is set when any of those ELTs has a
// non-zero loss for event i. An event with a clear bit contributes exactly
// zero to every layer of the group (absent losses are 0 and F_e(0) = 0 since
// D_e >= 0), so it is skipped without reading its row.
//
// Mapping: one warp per trial. The warp streams the trial's ids (coalesced,
// evict-first), tests each id's bit (the bitmap, C/8 bytes, stays in L1/L2),
// and appends the ids whose bit is set to a per-warp queue in shared memory.
// Each time 32 are queued, every lane takes one and evaluates it fully: one
// row read (np * 4 contiguous bytes, not allocated in L1 so the bitmap stays
// there), F_e per ELT in FP32, the per-layer ELT sums in the group's ELT
// order, the occurrence terms, and the occurrence-net loss added to the
// lane's per-layer aggregate. That aggregate is a compensated FP32 pair
// (Knuth's two-sum: the pair holds the exact sum up to a second-order term
// of order n u^2), folded into FP64 once per trial, so the FP64 pipe is used
// per trial rather than per event; the warp then reduces the lanes' FP64
// partials and applies the aggregate terms in FP64.
#include <limits>

#include "art_internal.cuh"

namespace art {

namespace {

constexpr int kSkipThreads = 256;
constexpr int kSkipWarps = kSkipThreads / 32;
#ifndef ART_SKIP_IDS_PER_LANE
#define ART_SKIP_IDS_PER_LANE 8
#endif
constexpr int kSkipIdsPerLane = ART_SKIP_IDS_PER_LANE;

__device__ __forceinline__ uint32_t ld_bitmap(const uint32_t* p) {
    uint32_t v;
    asm("ld.global.nc.L1::evict_last.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ float4 ld_row_no_l1(const float4* p) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}

// s + e += v without losing the rounding error of the FP32 add (two-sum).
__device__ __forceinline__ void two_sum_acc(float& s, float& e, float v) {
    const float t = s + v;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (v - bp);
    s = t;
    e += err;
}

template <int NP, int LT>
__device__ __forceinline__ void eval_event(const GroupArgs& g, int32_t id, float (&hi)[LT], float (&lo)[LT]) {
    const float4* row = reinterpret_cast<const float4*>(g.table) + (size_t)id * (NP / 4);
    float f[NP];
#pragma unroll
    for (int q = 0; q < NP / 4; ++q) {
        const float4 v = ld_row_no_l1(row + q);
        f[4 * q + 0] = fin_f32(v.x, g.m[4 * q + 0], g.d[4 * q + 0], g.lim[4 * q + 0]);
        f[4 * q + 1] = fin_f32(v.y, g.m[4 * q + 1], g.d[4 * q + 1], g.lim[4 * q + 1]);
        f[4 * q + 2] = fin_f32(v.z, g.m[4 * q + 2], g.d[4 * q + 2], g.lim[4 * q + 2]);
        f[4 * q + 3] = fin_f32(v.w, g.m[4 * q + 3], g.d[4 * q + 3], g.lim[4 * q + 3]);
    }
#pragma unroll
    for (int j = 0; j < LT; ++j) {
        float x = 0.0f;
#pragma unroll
        for (int k = 0; k < NP; ++k)
            if (g.member[j] & (1u << k)) x += f[k];
        const float o = xl_f32(x, g.occ_ret[j], g.occ_lim[j]);
        if (o > 0.0f) two_sum_acc(hi[j], lo[j], o);
    }
}

template <int NP, int LT>
__global__ void __launch_bounds__(kSkipThreads) ylt_skip_kernel(const GroupArgs g, const YetArgs y,
                                                               double* __restrict__ ylt,
                                                               uint8_t* __restrict__ branch,
                                                               int* __restrict__ flags) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int E = kSkipIdsPerLane;  // ids per lane per chunk: a chunk is 32 * E events
    __shared__ int32_t s_queue[kSkipWarps][64];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= y.n_trials) return;  // whole warp
    int32_t* q = s_queue[wib];
    const unsigned lt_mask = (1u << lane) - 1u;
    int64_t b, e;
    bool bad_off;
    trial_range(y, t, b, e, bad_off);
    float hi[LT], lo[LT];
#pragma unroll
    for (int j = 0; j < LT; ++j) {
        hi[j] = 0.0f;
        lo[j] = 0.0f;
    }
    bool bad_id = false;
    int qn = 0;  // warp-uniform queue length, < 32 between steps
    // the chunk's ids are all requested before any is used, and the next
    // chunk's ids are requested before this chunk's rows
    int32_t nid[E];
#pragma unroll
    for (int k = 0; k < E; ++k) {
        const int64_t d = b + k * 32 + lane;
        nid[k] = d < e ? ld_stream(y.ids + d) : -1;
    }
    for (int64_t d0 = b; d0 < e; d0 += 32 * E) {
        int32_t id[E];
#pragma unroll
        for (int k = 0; k < E; ++k) id[k] = nid[k];
        const int64_t d1 = d0 + 32 * E;
        if (d1 < e) {
#pragma unroll
            for (int k = 0; k < E; ++k) {
                const int64_t d = d1 + k * 32 + lane;
                nid[k] = d < e ? ld_stream(y.ids + d) : -1;
            }
        }
        uint32_t w[E];
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const bool live = d0 + k * 32 + lane < e;
            const bool ok = live && (unsigned)id[k] < (unsigned)y.catalogue;
            if (live && !ok) bad_id = true;
            w[k] = ok ? ld_bitmap(g.bitmap + (id[k] >> 5)) : 0u;
        }
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const bool nz = (w[k] >> (id[k] & 31)) & 1u;
            const unsigned m = __ballot_sync(FULL, nz);
            if (nz) q[qn + __popc(m & lt_mask)] = id[k];
            qn += __popc(m);
            if (qn >= 32) {
                __syncwarp();
                const int32_t mine = q[lane];
                const int32_t carry = q[32 + lane];
                __syncwarp();
                q[lane] = carry;  // entries 32 .. qn-1 move to the front
                qn -= 32;
                eval_event<NP, LT>(g, mine, hi, lo);
                __syncwarp();
            }
        }
    }
    __syncwarp();
    if (lane < qn) eval_event<NP, LT>(g, q[lane], hi, lo);
    if (bad_id) atomicOr(flags + kFlagIdRange, 1);
#pragma unroll
    for (int j = 0; j < LT; ++j) {
        double s = (double)hi[j] + (double)lo[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (lane == 0 && j < g.n_layers) {
            const size_t wi = (size_t)g.layer[j] * (size_t)y.n_trials + (size_t)t;
            ylt[wi] = xl_f64(s, g.agg_ret[j], g.agg_lim[j]);
            if (branch) branch[wi] = agg_branch(s, g.agg_ret[j], g.agg_lim[j]);
        }
    }
    if (lane == 0 && bad_off) atomicOr(flags + kFlagBadOffsets, 1);
}

template <int NP, int LT>
cudaError_t launch_group(const GroupArgs& g, const YetArgs& y, double* ylt, uint8_t* branch, int* flags,
                         cudaStream_t s) {
    auto kern = ylt_skip_kernel<NP, LT>;
    static bool configured = false;
    if (!configured) {
        // shared memory for the queues of six resident CTAs, the rest L1
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 10);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int64_t blocks = (y.n_trials + kSkipWarps - 1) / kSkipWarps;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    kern<<<(unsigned)blocks, kSkipThreads, 0, s>>>(g, y, ylt, branch, flags);
    return cudaGetLastError();
}

template <int NP>
cudaError_t launch_lt(const GroupArgs& g, const YetArgs& y, double* ylt, uint8_t* branch, int* flags,
                      cudaStream_t s) {
    if (g.n_layers <= 1) return launch_group<NP, 1>(g, y, ylt, branch, flags, s);
    if (g.n_layers <= 2) return launch_group<NP, 2>(g, y, ylt, branch, flags, s);
    if (g.n_layers <= 4) return launch_group<NP, 4>(g, y, ylt, branch, flags, s);
    return launch_group<NP, 8>(g, y, ylt, branch, flags, s);
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

cudaError_t launch_skip(art_portfolio* p, const YetArgs& y, double* ylt, uint8_t* branch, cudaStream_t s) {
    for (size_t gi = 0; gi < p->groups.size(); ++gi) {
        const GroupArgs& g = p->groups[gi];
        cudaError_t err;
        switch (p->group_np[gi]) {
            case 4: err = launch_lt<4>(g, y, ylt, branch, p->d_flags, s); break;
            case 8: err = launch_lt<8>(g, y, ylt, branch, p->d_flags, s); break;
            case 16: err = launch_lt<16>(g, y, ylt, branch, p->d_flags, s); break;
            case 24: err = launch_lt<24>(g, y, ylt, branch, p->d_flags, s); break;
            case 32: err = launch_lt<32>(g, y, ylt, branch, p->d_flags, s); break;
            default: err = cudaErrorInvalidValue;
        }
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

}  // namespace art

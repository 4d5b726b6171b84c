// ylt_plain.cu -- the plain one-layer-per-launch forward pass and the table
// builders (Section II, Algorithm 1; Section III, direct-access tables).
//
// Layout: each layer gets its own event-major direct-access table
// [C][np] FP32 (np = the layer's ELT count padded to 4, 8, 16, 24 or 32):
// row i holds event i's loss in each of the layer's ELTs, so one event's
// lookups for the whole layer are np * 4 contiguous bytes (one to four
// 32-byte sectors) instead of one sector per ELT. This is the paper's
// "ELTs combined as a single table" idea, gathered straight into registers
// rather than staged through shared memory.
//
// Mapping: one warp per trial, one lane per event (lane-strided, so each
// warp-wide id load is 128 coalesced bytes), U events per lane in flight.
// Per event the lane evaluates F_e on each ELT in FP32, sums in ELT order,
// applies the occurrence terms, and adds the result to its FP64 partial
// aggregate; the warp reduces the partials and lane 0 applies the aggregate
// terms (the telescoped form of Algorithm 1's running aggregate).
#include <limits>

#include "art_internal.cuh"

namespace art {

template <int NP, int U>
__global__ void __launch_bounds__(256) ylt_plain_kernel(const LayerArgs la, const YetArgs y,
                                                        double* __restrict__ ylt,
                                                        uint8_t* __restrict__ branch,
                                                        int* __restrict__ flags) {
    static_assert(NP % 4 == 0 && NP <= kMaxLayerElts, "row width");
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= y.n_trials) return;  // whole warp leaves together
    int64_t b, e;
    bool bad_off;
    trial_range(y, t, b, e, bad_off);
    const float4* __restrict__ tab = reinterpret_cast<const float4*>(la.table);
    double s = 0.0;
    bool bad_id = false;
    for (int64_t d0 = b; d0 < e; d0 += 32 * U) {
        int32_t id[U];
        bool live[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t d = d0 + u * 32 + lane;
            live[u] = d < e;
            id[u] = live[u] ? ld_stream(y.ids + d) : 0;
        }
        float4 r[U][NP / 4];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = live[u] && (unsigned)id[u] < (unsigned)y.catalogue;
            if (live[u] && !ok) bad_id = true;
            const float4* row = tab + (size_t)(ok ? id[u] : 0) * (NP / 4);
#pragma unroll
            for (int q = 0; q < NP / 4; ++q) r[u][q] = ok ? __ldg(row + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float x = 0.0f;
#pragma unroll
            for (int q = 0; q < NP / 4; ++q) {
                x += fin_f32(r[u][q].x, la.m[4 * q + 0], la.d[4 * q + 0], la.lim[4 * q + 0]);
                x += fin_f32(r[u][q].y, la.m[4 * q + 1], la.d[4 * q + 1], la.lim[4 * q + 1]);
                x += fin_f32(r[u][q].z, la.m[4 * q + 2], la.d[4 * q + 2], la.lim[4 * q + 2]);
                x += fin_f32(r[u][q].w, la.m[4 * q + 3], la.d[4 * q + 3], la.lim[4 * q + 3]);
            }
            const float o = xl_f32(x, la.occ_ret, la.occ_lim);
            if (o > 0.0f) s += (double)o;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (bad_id) atomicOr(flags + kFlagIdRange, 1);
    if (lane == 0) {
        if (bad_off) atomicOr(flags + kFlagBadOffsets, 1);
        const size_t w = (size_t)la.layer * (size_t)y.n_trials + (size_t)t;
        ylt[w] = xl_f64(s, la.agg_ret, la.agg_lim);
        if (branch) branch[w] = agg_branch(s, la.agg_ret, la.agg_lim);
    }
}

template <int NP, int U>
static cudaError_t launch_np(const LayerArgs& la, const YetArgs& y, double* ylt, uint8_t* branch, int* flags,
                             cudaStream_t s) {
    const int threads = 256;
    const int64_t warps_per_block = threads / 32;
    const int64_t blocks = (y.n_trials + warps_per_block - 1) / warps_per_block;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    ylt_plain_kernel<NP, U><<<(unsigned)blocks, threads, 0, s>>>(la, y, ylt, branch, flags);
    return cudaGetLastError();
}

cudaError_t launch_plain(art_portfolio* p, const YetArgs& y, double* ylt, uint8_t* branch, cudaStream_t s) {
    for (int32_t j = 0; j < p->n_layers; ++j) {
        LayerArgs la;
        la.table = p->layer_tab[j];
        const int32_t b = p->loff[j], n = p->loff[j + 1] - b;
        for (int k = 0; k < kMaxLayerElts; ++k) {
            if (k < n) {
                const int32_t e = p->lids[b + k];
                la.m[k] = p->mult[e];
                la.d[k] = p->ded[e];
                la.lim[k] = p->lim[e];
            } else {
                la.m[k] = 1.0f;
                la.d[k] = 0.0f;
                la.lim[k] = std::numeric_limits<float>::infinity();
            }
        }
        la.occ_ret = p->occ_ret[j];
        la.occ_lim = p->occ_lim[j];
        la.agg_ret = p->agg_ret[j];
        la.agg_lim = p->agg_lim[j];
        la.layer = j;
        cudaError_t err;
        if (p->flags & ART_FLAG_L2_PERSIST)
            set_window(s, la.table, sizeof(float) * (size_t)p->catalogue * p->layer_np[j]);
        switch (p->layer_np[j]) {
            case 4: err = launch_np<4, 8>(la, y, ylt, branch, p->d_flags, s); break;
            case 8: err = launch_np<8, 4>(la, y, ylt, branch, p->d_flags, s); break;
            case 16: err = launch_np<16, 4>(la, y, ylt, branch, p->d_flags, s); break;
            case 24: err = launch_np<24, 2>(la, y, ylt, branch, p->d_flags, s); break;
            case 32: err = launch_np<32, 2>(la, y, ylt, branch, p->d_flags, s); break;
            default: err = cudaErrorInvalidValue;
        }
        if (err != cudaSuccess) return err;
    }
    if (p->flags & ART_FLAG_L2_PERSIST) set_window(s, nullptr, 0);
    return cudaSuccess;
}

// Transpose-gather: dst[i][k] = src[elts[k]][i] for k < n, 0 for n <= k < np
// (elts == NULL means elts[k] = k). 32 x 32 tiles through shared memory so
// both the column reads and the row writes are coalesced.
__global__ void build_event_major_kernel(const float* __restrict__ src, int32_t catalogue,
                                         const int32_t* __restrict__ elts, int32_t n, int32_t np,
                                         float* __restrict__ dst32, double* __restrict__ dst64) {
    __shared__ float tile[32][33];
    const int64_t i0 = (int64_t)blockIdx.x * 32;
    const int k0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        const int k = k0 + r;
        const int64_t i = i0 + tx;
        float v = 0.0f;
        if (k < n && i < catalogue) {
            const int32_t e = elts ? elts[k] : k;
            v = src[(int64_t)e * catalogue + i];
        }
        tile[r][tx] = v;
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int64_t i = i0 + r;
        const int k = k0 + tx;
        if (i < catalogue && k < np) {
            if (dst32) dst32[i * np + k] = tile[tx][r];
            if (dst64) dst64[i * np + k] = (double)tile[tx][r];
        }
    }
}

cudaError_t build_layer_table(const float* src, int32_t catalogue, const int32_t* elts_dev, int32_t n, int32_t np,
                              float* dst, cudaStream_t s) {
    dim3 grid((unsigned)((catalogue + 31) / 32), (unsigned)((np + 31) / 32));
    build_event_major_kernel<<<grid, dim3(32, 8), 0, s>>>(src, catalogue, elts_dev, n, np, dst, nullptr);
    return cudaGetLastError();
}

cudaError_t build_pool_table(const float* src, int32_t catalogue, int32_t n_elt, int32_t np, float* dst32,
                             double* dst64, cudaStream_t s) {
    dim3 grid((unsigned)((catalogue + 31) / 32), (unsigned)((np + 31) / 32));
    build_event_major_kernel<<<grid, dim3(32, 8), 0, s>>>(src, catalogue, nullptr, n_elt, np, dst32, dst64);
    return cudaGetLastError();
}

}  // namespace art

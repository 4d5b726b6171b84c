// payouts.cu -- Algorithm 1's running form on the GPU for one layer: the
// cumulative aggregate C_d over a trial's events in trial order, the
// aggregate terms on every C_d, the per-event difference p_d = A(C_d) -
// A(C_{d-1}) (C_0 = 0: nothing is paid before the first event), and the
// position of the event that exhausts the aggregate limit (Section II: the
// aggregate terms apply to the cumulative sum, so the result depends on the
// sequence of prior events).
//
// Mapping: one warp per trial over the layer's event-major table; 32 events
// per step in trial order, lane l taking event d0 + l. Per event the lane
// forms x_d and o_d exactly as the forward kernels do (FP32, ELT order), then
// the warp scans o_d in FP64 (an inclusive shuffle scan) on top of the carry
// from the previous step, applies the aggregate terms to each C_d in FP64 and
// takes the difference with the previous event's value (the previous lane's,
// or the carried one). This path runs FP64 per event: it is a reporting path,
// not the throughput path.
#include <limits>

#include "art_internal.cuh"

namespace art {
namespace {

template <int NP>
__global__ void __launch_bounds__(256) payouts_kernel(const LayerArgs la, const YetArgs y,
                                                      double* __restrict__ payouts, int32_t* __restrict__ exhaust,
                                                      double* __restrict__ ylt, int* __restrict__ flags) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= y.n_trials) return;  // whole warp
    int64_t b, e;
    bool bad_off;
    trial_range(y, t, b, e, bad_off);
    const float4* __restrict__ tab = reinterpret_cast<const float4*>(la.table);
    double carry_c = 0.0, carry_a = 0.0;  // C and A(C) after the previous step
    int32_t first_cap = -1;
    bool bad_id = false;
    for (int64_t d0 = b; d0 < e; d0 += 32) {
        const int64_t d = d0 + lane;
        const bool live = d < e;
        const int32_t id = live ? ld_stream(y.ids + d) : 0;
        const bool ok = live && (unsigned)id < (unsigned)y.catalogue;
        if (live && !ok) bad_id = true;
        float x = 0.0f;
        if (ok) {
            const float4* row = tab + (size_t)id * (NP / 4);
#pragma unroll
            for (int q = 0; q < NP / 4; ++q) {
                const float4 r = __ldg(row + q);
                x += fin_f32(r.x, la.m[4 * q + 0], la.d[4 * q + 0], la.lim[4 * q + 0]);
                x += fin_f32(r.y, la.m[4 * q + 1], la.d[4 * q + 1], la.lim[4 * q + 1]);
                x += fin_f32(r.z, la.m[4 * q + 2], la.d[4 * q + 2], la.lim[4 * q + 2]);
                x += fin_f32(r.w, la.m[4 * q + 3], la.d[4 * q + 3], la.lim[4 * q + 3]);
            }
        }
        const double o = live ? (double)xl_f32(x, la.occ_ret, la.occ_lim) : 0.0;
        // inclusive scan of o over the lanes, in trial order
        double c = o;
#pragma unroll
        for (int k = 1; k < 32; k <<= 1) {
            const double v = __shfl_up_sync(FULL, c, k);
            if (lane >= k) c += v;
        }
        c += carry_c;
        const double a = xl_f64(c, la.agg_ret, la.agg_lim);
        double a_prev = __shfl_up_sync(FULL, a, 1);
        if (lane == 0) a_prev = carry_a;
        if (live && payouts) payouts[d] = a - a_prev;
        // the aggregate limit is exhausted at the first event whose C_d - AggR reaches AggL
        const unsigned capped = __ballot_sync(FULL, live && (c - la.agg_ret >= la.agg_lim));
        if (first_cap < 0 && capped) first_cap = (int32_t)(d0 - b) + __ffs(capped) - 1;
        carry_c = __shfl_sync(FULL, c, 31);
        carry_a = __shfl_sync(FULL, a, 31);
    }
    if (bad_id) atomicOr(flags + kFlagIdRange, 1);
    if (lane == 0) {
        if (bad_off) atomicOr(flags + kFlagBadOffsets, 1);
        if (exhaust) exhaust[t] = first_cap;
        if (ylt) ylt[t] = carry_a;  // A(C_K): the telescoped sum of the payouts
    }
}

template <int NP>
cudaError_t launch(const LayerArgs& la, const YetArgs& y, double* payouts, int32_t* exhaust, double* ylt, int* flags,
                   cudaStream_t s) {
    const int64_t blocks = (y.n_trials + 7) / 8;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    payouts_kernel<NP><<<(unsigned)blocks, 256, 0, s>>>(la, y, payouts, exhaust, ylt, flags);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_payouts(art_portfolio* p, int32_t j, const YetArgs& y, double* payouts, int32_t* exhaust,
                           double* ylt, cudaStream_t s) {
    if (y.n_trials == 0) return cudaSuccess;
    LayerArgs la;
    la.table = p->layer_tab[j];
    const int32_t b = p->loff[j], n = p->loff[j + 1] - b;
    for (int k = 0; k < kMaxLayerElts; ++k) {
        const bool real = k < n;
        const int32_t e = real ? p->lids[b + k] : 0;
        la.m[k] = real ? p->mult[e] : 1.0f;
        la.d[k] = real ? p->ded[e] : 0.0f;
        la.lim[k] = real ? p->lim[e] : std::numeric_limits<float>::infinity();
    }
    la.occ_ret = p->occ_ret[j];
    la.occ_lim = p->occ_lim[j];
    la.agg_ret = p->agg_ret[j];
    la.agg_lim = p->agg_lim[j];
    la.layer = j;
    switch (p->layer_np[j]) {
        case 4: return launch<4>(la, y, payouts, exhaust, ylt, p->d_flags, s);
        case 8: return launch<8>(la, y, payouts, exhaust, ylt, p->d_flags, s);
        case 16: return launch<16>(la, y, payouts, exhaust, ylt, p->d_flags, s);
        case 24: return launch<24>(la, y, payouts, exhaust, ylt, p->d_flags, s);
        case 32: return launch<32>(la, y, payouts, exhaust, ylt, p->d_flags, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace art

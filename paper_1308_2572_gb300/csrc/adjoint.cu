// adjoint.cu -- gradient of sum_{j,t} g_{j,t} Y_{j,t} with respect to the
// layer terms and the ELT loss multipliers (the pricing sensitivity; the
// paper has no gradients, it is added around Section II's Algorithm 1).
//
// Y = A(S), S = sum_d O(x_d), x_d = sum_e F_e(l_e[E_d]) is piecewise linear
// in every term. With a = [branch == mid] and c = [branch == capped] read
// from the forward's aggregate branch code:
//   dY/dAggR = -a, dY/dAggL = c,
//   dY/dOccR = -a #{d : OccR < x_d < OccR + OccL},
//   dY/dOccL =  a #{d : x_d > OccR + OccL},
//   dY/dm_e  =  a sum_d [o_d mid][D_e < m_e l < D_e + Lim_e] l.
// Only trials with a != 0 and g != 0 are re-read; their per-event branches
// are recomputed with exactly the forward's FP32 arithmetic (same F, same ELT
// order, same occurrence subtraction), so they match the forward bit for bit.
//
// Mapping: the plain forward's (warp per trial, lane per event), over a
// persistent grid with a static trial stride. Within a trial each lane counts
// its events on the middle and capped occurrence branches (integers) and sums
// the losses l of each ELT's middle-branch events as a compensated FP32 pair
// (two-sum, exact to second order); at the end of the trial these are scaled
// by the trial's weight g into FP64 accumulators, so FP64 arithmetic runs per
// trial, not per event (the FP64 pipe of this part is slow). The FP64 sums
// are reduced warp -> CTA -> grid in a fixed order (deterministic).
#include <limits>

#include "art_internal.cuh"

namespace art {

namespace {

constexpr int kAdjThreads = 256;

__device__ __forceinline__ void two_sum_add(float& s, float& e, float v) {
    const float t = s + v;
    const float bp = t - s;
    e += (s - (t - bp)) + (v - bp);
    s = t;
}

template <int NP, int U>
__global__ void __launch_bounds__(kAdjThreads) adjoint_kernel(const LayerArgs la, const YetArgs y,
                                                              const uint8_t* __restrict__ branch,
                                                              const double* __restrict__ g,
                                                              double* __restrict__ partial) {
    constexpr int W = 4 + NP;  // OccR, OccL, AggR, AggL, then the layer's ELT slots
    __shared__ double sh[kAdjThreads / 32][W];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float4* __restrict__ tab = reinterpret_cast<const float4*>(la.table);
    double acc_or = 0.0, acc_ol = 0.0, acc_ar = 0.0, acc_al = 0.0;
    double acc_m[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc_m[k] = 0.0;

    for (int64_t t = warp0; t < y.n_trials; t += n_warps) {
        const size_t w = (size_t)la.layer * (size_t)y.n_trials + (size_t)t;
        const uint8_t code = branch[w];
        const double gt = g[w];
        if (gt == 0.0) continue;
        if (code == 2) {
            if (lane == 0) acc_al += gt;
            continue;
        }
        if (code != 1) continue;
        if (lane == 0) acc_ar -= gt;
        int64_t b, e;
        bool bad_off;
        trial_range(y, t, b, e, bad_off);
        int n_mid = 0, n_cap = 0;
        float mh[NP], ml[NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            mh[k] = 0.0f;
            ml[k] = 0.0f;
        }
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
                const float4* row = tab + (size_t)(ok ? id[u] : 0) * (NP / 4);
#pragma unroll
                for (int q = 0; q < NP / 4; ++q) r[u][q] = ok ? __ldg(row + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float v[NP];
#pragma unroll
                for (int q = 0; q < NP / 4; ++q) {
                    v[4 * q + 0] = r[u][q].x;
                    v[4 * q + 1] = r[u][q].y;
                    v[4 * q + 2] = r[u][q].z;
                    v[4 * q + 3] = r[u][q].w;
                }
                float x = 0.0f;
#pragma unroll
                for (int k = 0; k < NP; ++k) x += fin_f32(v[k], la.m[k], la.d[k], la.lim[k]);
                const float wo = x - la.occ_ret;  // the forward's occurrence subtraction
                const bool mid = wo > 0.0f && wo < la.occ_lim;
                const bool cap = wo > la.occ_lim;
                n_cap += cap ? 1 : 0;
                if (mid) {
                    ++n_mid;
#pragma unroll
                    for (int k = 0; k < NP; ++k) {
                        const float wf = __fmaf_rn(la.m[k], v[k], -la.d[k]);
                        if (wf > 0.0f && wf < la.lim[k]) two_sum_add(mh[k], ml[k], v[k]);
                    }
                }
            }
        }
        // once per trial: the lane's counts and sums, weighted by g, in FP64
        acc_or -= gt * (double)n_mid;
        acc_ol += gt * (double)n_cap;
#pragma unroll
        for (int k = 0; k < NP; ++k) acc_m[k] += gt * ((double)mh[k] + (double)ml[k]);
    }
    // warp -> CTA -> grid partial, fixed order
    double vals[W];
    vals[0] = acc_or;
    vals[1] = acc_ol;
    vals[2] = acc_ar;
    vals[3] = acc_al;
#pragma unroll
    for (int k = 0; k < NP; ++k) vals[4 + k] = acc_m[k];
#pragma unroll
    for (int i = 0; i < W; ++i) {
        double v = vals[i];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) sh[wib][i] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        double s = 0.0;
        for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += sh[wv][i];
        partial[(size_t)blockIdx.x * W + i] = s;
    }
}

// Sum the per-CTA partials of one layer in order into layer_grad[j][4 + 32].
__global__ void reduce_partials_kernel(const double* __restrict__ partial, int nblk, int width, int layer,
                                       double* __restrict__ layer_grad) {
    const int i = threadIdx.x;
    if (i >= width) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * width + i];
    layer_grad[(size_t)layer * (4 + kMaxLayerElts) + i] = s;
}

// grad_terms[j][0..3] and grad_mult[e] = sum over layers (in order) of the
// layer's slot sums for ELT e.
__global__ void scatter_grad_kernel(const double* __restrict__ layer_grad, int n_layers, int n_elt,
                                    const int32_t* __restrict__ loff, const int32_t* __restrict__ lids,
                                    double* __restrict__ grad_terms, double* __restrict__ grad_mult) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_layers * 4) grad_terms[i] = layer_grad[(size_t)(i / 4) * (4 + kMaxLayerElts) + (i % 4)];
    if (i < n_elt) {
        double s = 0.0;
        for (int j = 0; j < n_layers; ++j)
            for (int c = loff[j]; c < loff[j + 1]; ++c)
                if (lids[c] == i) s += layer_grad[(size_t)j * (4 + kMaxLayerElts) + 4 + (c - loff[j])];
        grad_mult[i] = s;
    }
}

template <int NP, int U>
cudaError_t launch_layer(const LayerArgs& la, const YetArgs& y, const uint8_t* branch, const double* g,
                         double* partial, int nblk, double* layer_grad, cudaStream_t s) {
    adjoint_kernel<NP, U><<<nblk, kAdjThreads, 0, s>>>(la, y, branch, g, partial);
    cudaError_t err = cudaGetLastError();
    if (err) return err;
    reduce_partials_kernel<<<1, 64, 0, s>>>(partial, nblk, 4 + NP, la.layer, layer_grad);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adjoint(art_portfolio* p, const YetArgs& y, const uint8_t* branch, const double* g,
                           double* grad_terms, double* grad_mult, cudaStream_t s) {
    int per_sm = 4;
    const int nblk = p->num_sms * per_sm;
    const size_t lg_bytes = sizeof(double) * (size_t)p->n_layers * (4 + kMaxLayerElts);
    const size_t part_bytes = sizeof(double) * (size_t)nblk * (4 + kMaxLayerElts);
    char* w = nullptr;
    cudaError_t err = cudaMallocAsync((void**)&w, lg_bytes + part_bytes + 256, s);
    if (err) return err;
    double* layer_grad = (double*)w;
    double* partial = (double*)(w + ((lg_bytes + 255) & ~(size_t)255));
    do {
        if ((err = cudaMemsetAsync(layer_grad, 0, lg_bytes, s))) break;
        if (y.n_trials > 0) {
            for (int32_t j = 0; j < p->n_layers && !err; ++j) {
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
                    case 4: err = launch_layer<4, 4>(la, y, branch, g, partial, nblk, layer_grad, s); break;
                    case 8: err = launch_layer<8, 2>(la, y, branch, g, partial, nblk, layer_grad, s); break;
                    case 16: err = launch_layer<16, 1>(la, y, branch, g, partial, nblk, layer_grad, s); break;
                    case 24: err = launch_layer<24, 1>(la, y, branch, g, partial, nblk, layer_grad, s); break;
                    case 32: err = launch_layer<32, 1>(la, y, branch, g, partial, nblk, layer_grad, s); break;
                    default: err = cudaErrorInvalidValue;
                }
            }
            if (err) break;
        }
        const int n_out = p->n_layers * 4 > p->n_elt ? p->n_layers * 4 : p->n_elt;
        scatter_grad_kernel<<<(n_out + 127) / 128, 128, 0, s>>>(layer_grad, p->n_layers, p->n_elt, p->d_loff, p->d_lids,
                                                               grad_terms, grad_mult);
        err = cudaGetLastError();
    } while (0);
    const cudaError_t e2 = cudaFreeAsync(w, s);
    return err ? err : e2;
}

}  // namespace art

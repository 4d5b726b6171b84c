// shard.cu -- metrics of a YLT whose trials are split between GPUs (Section
// III: trials are independent; Section IV-C: the multi-GPU runs split the
// trials of the YET between the GPUs, each computing its trials' losses).
//
// PML_p and TVaR_p of a layer depend only on its k largest trial losses,
// k = ceil((1 - p) N), and the layer's k largest losses over all trials are
// among the union of every shard's k largest. So each shard reduces its YLT
// rows to a top-k list and a loss sum (art_topk, on its GPU), the lists are
// gathered, and the merge selects exactly from their union (art_merge_topk,
// on the host): the same PML bits as one GPU holding every trial, and the
// same TVaR and mean up to the order of the FP64 additions.
//
// A shard's list is written in the order of the trials (values above the
// shard's k-th largest, by a count, a scan and a write at fixed block
// ranges), then the k-th largest itself as often as it is needed, then zeros
// (a shard with fewer than k trials): the same list for the same YLT, call
// after call. The merge sums the union in the order of the shards and their
// lists, so its results are deterministic too.
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "art_internal.cuh"

namespace art {
namespace {

constexpr int kTopThreads = 256;

__device__ __forceinline__ unsigned long long abs_key(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

// Block b of layer j covers trials [b * per, min(n, (b + 1) * per)) and counts
// those whose loss lies above the layer's threshold key.
__global__ void __launch_bounds__(kTopThreads) topk_count_kernel(const double* __restrict__ ylt, int64_t n,
                                                                 int64_t per, const double* __restrict__ thr,
                                                                 unsigned long long* __restrict__ cnt) {
    __shared__ unsigned long long sh[kTopThreads / 32];
    const int j = blockIdx.y;
    const unsigned long long t = abs_key(thr[j]);
    const double* row = ylt + (size_t)j * (size_t)n;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(n, b0 + per);
    unsigned long long c = 0;
    for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) c += abs_key(__ldcs(row + i)) > t ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0;
        for (int w = 0; w < kTopThreads / 32; ++w) s += sh[w];
        cnt[(size_t)j * gridDim.x + blockIdx.x] = s;
    }
}

// Writes block b's losses above the threshold at its offset (the counts of
// the blocks before it), in trial order, then its share of the tail of the
// list: the threshold value up to k_eff, zeros up to k.
__global__ void __launch_bounds__(kTopThreads) topk_write_kernel(const double* __restrict__ ylt, int64_t n,
                                                                 int64_t per, const double* __restrict__ thr,
                                                                 const unsigned long long* __restrict__ cnt,
                                                                 int64_t k, int64_t k_eff,
                                                                 double* __restrict__ top) {
    __shared__ unsigned long long sh_off, sh_total;
    __shared__ unsigned int sh_warp[kTopThreads / 32];
    const int j = blockIdx.y;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const unsigned long long* cj = cnt + (size_t)j * gridDim.x;
    if (threadIdx.x == 0) {
        unsigned long long off = 0, total = 0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            if (b == blockIdx.x) off = total;
            total += cj[b];
        }
        sh_off = off;
        sh_total = total;
    }
    __syncthreads();
    const double tv = thr[j];
    const unsigned long long t = abs_key(tv);
    const double* row = ylt + (size_t)j * (size_t)n;
    double* out = top + (size_t)j * (size_t)k;
    const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(n, b0 + per);
    unsigned long long base = sh_off;
    for (int64_t i0 = b0; i0 < b1; i0 += blockDim.x) {
        const int64_t i = i0 + threadIdx.x;
        const unsigned long long key = i < b1 ? abs_key(__ldcs(row + i)) : 0ULL;
        const bool up = i < b1 && key > t;
        const unsigned m = __ballot_sync(0xffffffffu, up);
        if (lane == 0) sh_warp[wib] = __popc(m);
        __syncthreads();
        unsigned long long before = 0, step = 0;
        for (int w = 0; w < kTopThreads / 32; ++w) {
            if (w < wib) before += sh_warp[w];
            step += sh_warp[w];
        }
        const unsigned long long slot = base + before + __popc(m & ((1u << lane) - 1u));
        if (up && slot < (unsigned long long)k) out[slot] = __longlong_as_double((long long)key);
        base += step;
        __syncthreads();
    }
    // the tail of the list, shared out between the layer's blocks
    const unsigned long long total = min(sh_total, (unsigned long long)k_eff);
    for (int64_t s = (int64_t)total + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < k;
         s += (int64_t)gridDim.x * blockDim.x)
        out[s] = s < k_eff ? __longlong_as_double((long long)t) : 0.0;
}

}  // namespace
}  // namespace art

using namespace art;

extern "C" art_status art_topk(const double* ylt_dev, int64_t n_trials, int32_t n_layers, int64_t k,
                               double* top_dev, double* sum_dev, cudaStream_t stream) {
    if (!ylt_dev || !top_dev || n_trials < 1 || n_trials > 0x7fffffffLL || n_layers < 1 || n_layers > 65535 ||
        k < 1 || k > 0x7fffffffLL)
        return ART_EINVAL;
    const int64_t k_eff = std::min(k, n_trials);
    int dev = 0, sms = 148;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) {
        set_last_error(e);
        return ART_ECUDA;
    }
    // blocks per layer: about 8 per SM over all layers, at least 4096 trials each
    const int64_t want = std::max<int64_t>(1, std::min<int64_t>((8LL * sms + n_layers - 1) / n_layers,
                                                                (n_trials + 4095) / 4096));
    const int64_t per = (n_trials + want - 1) / want;
    const int nblk = (int)((n_trials + per - 1) / per);
    double* thr = nullptr;
    unsigned long long* cnt = nullptr;
    const size_t thr_bytes = (sizeof(double) * (size_t)n_layers + 255) & ~(size_t)255;
    if ((e = cudaMallocAsync((void**)&thr, thr_bytes + sizeof(unsigned long long) * (size_t)n_layers * nblk, stream))) {
        set_last_error(e);
        return ART_ECUDA;
    }
    cnt = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(thr) + thr_bytes);
    // the k_eff-th largest loss of every layer, and the layer sums
    const int64_t kk = k_eff;
    e = metrics_run_k(ylt_dev, n_trials, n_layers, &kk, 1, nullptr, thr, nullptr, sum_dev, stream);
    if (!e) {
        topk_count_kernel<<<dim3(nblk, n_layers), kTopThreads, 0, stream>>>(ylt_dev, n_trials, per, thr, cnt);
        e = cudaGetLastError();
    }
    if (!e) {
        topk_write_kernel<<<dim3(nblk, n_layers), kTopThreads, 0, stream>>>(ylt_dev, n_trials, per, thr, cnt, k,
                                                                           k_eff, top_dev);
        e = cudaGetLastError();
    }
    const cudaError_t e2 = cudaFreeAsync(thr, stream);
    if (e || e2) {
        set_last_error(e ? e : e2);
        return ART_ECUDA;
    }
    return ART_OK;
}

extern "C" art_status art_merge_topk(const double* top_host, const double* sum_host, int32_t n_shards,
                                     int32_t n_layers, int64_t k, int64_t n_trials_total, const double* probs_host,
                                     int32_t n_p, double* mean_host, double* pml_host, double* tvar_host) {
    if (!top_host || !sum_host || n_shards < 1 || n_layers < 1 || k < 1 || n_trials_total < 1 || !probs_host ||
        n_p < 1 || n_p > kMaxProbs)
        return ART_EINVAL;
    if ((double)n_shards * (double)n_layers * (double)k > 1e10) return ART_EINVAL;
    int64_t kq[kMaxProbs];
    for (int q = 0; q < n_p; ++q) {
        if (!(probs_host[q] > 0.0 && probs_host[q] < 1.0)) return ART_EINVAL;
        kq[q] = tail_count(probs_host[q], n_trials_total);
        if (kq[q] > k) return ART_EINVAL;  // the lists are too short for this probability
    }
    const int64_t u = (int64_t)n_shards * k;
    auto layer = [&](int32_t j, std::vector<double>& all, std::vector<double>& work) {
        // the union of the shards' lists, in shard order
        for (int32_t s = 0; s < n_shards; ++s) {
            const double* src = top_host + ((size_t)s * n_layers + j) * (size_t)k;
            std::copy(src, src + k, all.begin() + (size_t)s * k);
        }
        if (mean_host) {
            double m = 0.0;
            for (int32_t s = 0; s < n_shards; ++s) m += sum_host[(size_t)s * n_layers + j];
            mean_host[j] = m / (double)n_trials_total;
        }
        for (int q = 0; q < n_p; ++q) {
            work = all;
            std::nth_element(work.begin(), work.begin() + (kq[q] - 1), work.end(), std::greater<double>());
            const double v = work[kq[q] - 1];
            double s = 0.0;
            int64_t c = 0;
            for (int64_t i = 0; i < u; ++i)
                if (all[i] > v) {
                    s += all[i];
                    ++c;
                }
            if (pml_host) pml_host[(size_t)j * n_p + q] = v;
            if (tvar_host) tvar_host[(size_t)j * n_p + q] = (s + (double)(kq[q] - c) * v) / (double)kq[q];
        }
    };
    const int32_t n_threads =
        (int32_t)std::max<int64_t>(1, std::min<int64_t>({(int64_t)std::thread::hardware_concurrency(), n_layers,
                                                         (int64_t)16}));
    std::vector<std::thread> pool;
    for (int32_t w = 0; w < n_threads; ++w)
        pool.emplace_back([&, w] {
            std::vector<double> all((size_t)u), work((size_t)u);
            for (int32_t j = w; j < n_layers; j += n_threads) layer(j, all, work);
        });
    for (auto& t : pool) t.join();
    return ART_OK;
}

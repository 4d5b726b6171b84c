// metrics.cu -- expected loss, PML and TVaR from the YLT (Section I names PML
// and TVaR as the risk metrics derived from a YLT; Section II applies
// "financial functions or filters" to the trial losses).
//
// Reading: per layer, with k = ceil((1-p) N) (at least 1), PML_p is the k-th
// largest trial loss and TVaR_p the mean of the k largest.
//
// Exact selection without a sort: trial losses are >= 0, so the FP64 bit
// pattern (sign cleared, which also folds -0 onto +0) orders like the value. A
// most-significant-digit radix select over 63 bits in six passes (digits of
// 11, 11, 11, 11, 11 and 8 bits) narrows, for every (layer, probability)
// problem at once, the prefix of the k-th largest key. Each pass is one
// launch: its blocks histogram the keys that match the prefix found so far
// (shared-memory histograms with warp-aggregated atomics: lanes holding the
// same digit add once; flushed to global with atomics), and the last block of
// each layer to finish (a ticket counter after a fence; no block waits for
// another) picks the digit where the count from the top crosses the remaining
// rank. Problems of a layer that share a prefix (all of them in the first
// pass) share one histogram, and a problem whose candidates all hold one key
// (their smallest and largest agree) is decided at once, its later passes
// returning early. A last launch sums the values strictly above the k-th
// largest, and its last block reduces the partials: TVaR adds the tied
// remainder, (sum_gt + (k - count_gt) * PML) / k. Seven launches in all. Sums
// are FP64 and deterministic (per-thread, per-block, then per-problem in a
// fixed order).
#include <algorithm>
#include <cmath>

#include "art_internal.cuh"

namespace art {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;  // values per thread whose loads are in flight together
constexpr int kMaxBins = 2048;
constexpr int kPasses = 6;
__host__ __device__ constexpr int pass_shift(int i) { return i < 5 ? 52 - 11 * i : 0; }
__host__ __device__ constexpr int pass_bits(int i) { return i < 5 ? 11 : 8; }

struct KParams {
    long long k[kMaxProbs];
};

struct SelState {
    unsigned long long prefix;
    unsigned long long mask;
    long long krem;
    long long k;
};

__device__ __forceinline__ unsigned long long key_of(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

// A problem whose mask covers every key bit is decided: its prefix is the key.
constexpr unsigned long long kAllKeyBits = 0x7fffffffffffffffULL;

// Block-wide maximum of a 64-bit value (valid in thread 0).
__device__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* sh) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    unsigned long long r = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = max(r, sh[i]);
    return r;
}

// Block-wide sum of a double in a fixed order (warp tree, then warps in order).
__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    return r;  // valid in thread 0
}

__device__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    unsigned long long r = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    return r;
}

// Backward: counts of values above and equal to each PML, then the weights.
template <int NQ>
__global__ void __launch_bounds__(kThreads) count_kernel(const double* __restrict__ ylt, int64_t n, int n_p,
                                                         const double* __restrict__ pml,
                                                         unsigned long long* __restrict__ part_gt,
                                                         unsigned long long* __restrict__ part_eq) {
    __shared__ unsigned long long sh_red_u[32];
    const int j = blockIdx.y;
    unsigned long long thr[NQ], gt[NQ], eq[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        thr[q] = q < n_p ? key_of(pml[j * n_p + q]) : 0;
        gt[q] = 0;
        eq[q] = 0;
    }
    const double* row = ylt + (size_t)j * (size_t)n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = key_of(row[i]);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            gt[q] += (q < n_p && key > thr[q]) ? 1 : 0;
            eq[q] += (q < n_p && key == thr[q]) ? 1 : 0;
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (q >= n_p) break;
        const unsigned long long a = block_sum_u64(gt[q], sh_red_u);
        const unsigned long long b = block_sum_u64(eq[q], sh_red_u);
        if (threadIdx.x == 0) {
            const size_t w = ((size_t)j * n_p + q) * gridDim.x + blockIdx.x;
            part_gt[w] = a;
            part_eq[w] = b;
        }
    }
}

__global__ void weights_kernel(int n_layers, int n_p, int nblk, const KParams kq,
                               const unsigned long long* __restrict__ part_gt,
                               const unsigned long long* __restrict__ part_eq, double* __restrict__ w_gt,
                               double* __restrict__ w_eq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_layers * n_p) return;
    unsigned long long cg = 0, ce = 0;
    for (int b = 0; b < nblk; ++b) {
        cg += part_gt[(size_t)i * nblk + b];
        ce += part_eq[(size_t)i * nblk + b];
    }
    const double k = (double)kq.k[i % n_p];
    w_gt[i] = 1.0 / k;
    w_eq[i] = ce ? ((k - (double)cg) / (k * (double)ce)) : 0.0;
}

template <int NQ>
__global__ void __launch_bounds__(kThreads) grad_ylt_kernel(const double* __restrict__ ylt, int64_t n, int n_p,
                                                            const double* __restrict__ pml,
                                                            const double* __restrict__ gmean,
                                                            const double* __restrict__ gtvar,
                                                            const double* __restrict__ w_gt,
                                                            const double* __restrict__ w_eq,
                                                            double* __restrict__ gylt) {
    const int j = blockIdx.y;
    const double base = gmean ? gmean[j] / (double)n : 0.0;
    unsigned long long thr[NQ];
    double cg[NQ], ce[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const bool on = q < n_p && gtvar;
        thr[q] = on ? key_of(pml[j * n_p + q]) : 0;
        cg[q] = on ? gtvar[j * n_p + q] * w_gt[j * n_p + q] : 0.0;
        ce[q] = on ? gtvar[j * n_p + q] * w_eq[j * n_p + q] : 0.0;
    }
    const double* row = ylt + (size_t)j * (size_t)n;
    double* out = gylt + (size_t)j * (size_t)n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = key_of(row[i]);
        double g = base;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if (q < n_p) {
                if (key > thr[q]) g += cg[q];
                else if (key == thr[q]) g += ce[q];
            }
        }
        out[i] = g;
    }
}

// Digit pick of one (layer, probability) problem by the whole block: the
// digit where the count of keys from the top reaches the remaining rank;
// extends the prefix, clears the problem's bins. Histogram reads bypass L1
// (the bins were filled by other blocks' atomics).
__device__ void select_block(SelState* __restrict__ st, unsigned int* __restrict__ h, int shift, int bits,
                             bool first, long long k0) {
    __shared__ unsigned int sh_bins[kMaxBins];
    __shared__ unsigned long long sh_scan[kThreads];
    __shared__ int sh_bin;
    __shared__ unsigned long long sh_above;
    const int nb = 1 << bits;
    const int per = nb / kThreads > 0 ? nb / kThreads : 1;
    const long long krem = first ? k0 : st->krem;
    // every bin requested at once (8 per thread), then cleared for the next pass
#pragma unroll
    for (int r = 0; r < kMaxBins / kThreads; ++r) {
        const int i = r * kThreads + threadIdx.x;
        if (i < nb) sh_bins[i] = __ldcg(h + i);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
    // thread i covers descending ranks [i*per, (i+1)*per): bins nb-1-i*per downwards
    unsigned long long local = 0;
    if (threadIdx.x * per < nb)
        for (int r = 0; r < per; ++r) local += sh_bins[nb - 1 - (threadIdx.x * per + r)];
    sh_scan[threadIdx.x] = local;
    if (threadIdx.x == 0) sh_bin = -1;
    __syncthreads();
    for (int o = 1; o < kThreads; o <<= 1) {
        const unsigned long long add = threadIdx.x >= (unsigned)o ? sh_scan[threadIdx.x - o] : 0ULL;
        __syncthreads();
        sh_scan[threadIdx.x] += add;
        __syncthreads();
    }
    const unsigned long long incl = sh_scan[threadIdx.x];
    const unsigned long long excl = incl - local;
    if (threadIdx.x * per < nb && (long long)excl < krem && krem <= (long long)incl) {
        unsigned long long run = excl;
        for (int r = 0; r < per; ++r) {
            const int bin = nb - 1 - (threadIdx.x * per + r);
            const unsigned c = sh_bins[bin];
            if ((long long)(run + c) >= krem) {
                sh_bin = bin;
                sh_above = run;
                break;
            }
            run += c;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int bin = sh_bin < 0 ? 0 : sh_bin;  // unreachable when counts are consistent
        const unsigned long long prefix = first ? 0ULL : st->prefix, mask = first ? 0ULL : st->mask;
        st->prefix = prefix | (unsigned long long)bin << shift;
        st->mask = mask | (unsigned long long)(nb - 1) << shift;
        st->krem = krem - (long long)(sh_bin < 0 ? 0 : sh_above);
        if (first) st->k = k0;
    }
    __syncthreads();
}

// One radix pass fused with its digit pick: grid (blocks_per_layer,
// n_layers). Every block histograms its keys (as hist_kernel) and flushes
// them with atomics; the last block of a layer to finish (a ticket counter,
// after a fence: no block waits for another) picks the digits of the
// layer's problems and resets the counter. The first pass matches every key
// (it starts the state from k) and writes the blocks' partial sums (mean).
template <int NQ>
__global__ void __launch_bounds__(kThreads) hist_select_kernel(const double* __restrict__ ylt, int64_t n, int n_p,
                                                               SelState* __restrict__ st, int shift, int bits,
                                                               bool first, const KParams kq,
                                                               unsigned int* __restrict__ ghist,
                                                               unsigned long long* __restrict__ minmax,
                                                               double* __restrict__ part_sum,
                                                               unsigned int* __restrict__ tickets) {
    extern __shared__ unsigned int sh_hist[];  // [n_p][1 << bits]
    __shared__ double sh_red[32];
    __shared__ unsigned long long sh_red_u[32];
    __shared__ bool sh_last;
    const int nb = 1 << bits;
    const int j = blockIdx.y;
    unsigned long long pre[NQ], msk[NQ];
    bool done[NQ];
    bool all_done = true;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        pre[q] = q < n_p ? (first ? 0ULL : st[j * n_p + q].prefix) : 1ULL;  // unused slots never match
        msk[q] = q < n_p ? (first ? 0ULL : st[j * n_p + q].mask) : 0ULL;
        done[q] = q >= n_p || msk[q] == kAllKeyBits;  // decided by an earlier pass
        all_done = all_done && done[q];
    }
    if (all_done) return;  // the same for every block of the layer: no ticket is taken
    // problems with the same prefix and mask see the same candidates (every
    // problem in the first pass; later, probabilities whose k-th largest
    // keys share their leading digits): the first of them, the source,
    // histograms for all
    __shared__ int sh_src[kMaxProbs];
    int src[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        src[q] = q;
#pragma unroll
        for (int r = NQ - 1; r >= 0; --r)
            if (r < q && !done[r] && !done[q] && pre[r] == pre[q] && msk[r] == msk[q]) src[q] = r;
        if (threadIdx.x == 0 && q < n_p) sh_src[q] = src[q];
    }
    for (int i = threadIdx.x; i < n_p * nb; i += blockDim.x) sh_hist[i] = 0;
    // largest candidate key and largest complement (the smallest candidate)
    unsigned long long kmax[NQ], kinv[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        kmax[q] = 0;
        kinv[q] = 0;
    }
    __syncthreads();
    const double* row = ylt + (size_t)j * (size_t)n;
    double sum = 0.0;
    const unsigned dmask = (unsigned)nb - 1u;
    const unsigned lane = threadIdx.x & 31;
    // kUnroll values per thread per step, their loads issued together
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kUnroll; i0 < n;
         i0 += (int64_t)gridDim.x * blockDim.x * kUnroll) {
        double v[kUnroll];
        bool valid[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x + threadIdx.x;
            valid[u] = i < n;
            v[u] = valid[u] ? row[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (first) sum += v[u];
            const unsigned long long key = key_of(v[u]);
            const unsigned dig = (unsigned)(key >> shift) & dmask;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                if (q < n_p && !done[q] && src[q] == q) {  // the same for the whole block
                    const bool hit = valid[u] && (key & msk[q]) == pre[q];
                    // after the first pass few warps hold a candidate at all
                    if (first || __any_sync(0xffffffffu, hit)) {
                        // lanes with the same digit add once (losses cluster:
                        // many trials share a value, such as a capped layer's AggL)
                        const unsigned peers = __match_any_sync(0xffffffffu, hit ? dig : 0xffffffffu);
                        if (hit && lane == (unsigned)(__ffs(peers) - 1))
                            atomicAdd(&sh_hist[q * nb + dig], __popc(peers));
                        if (hit) {
                            kmax[q] = max(kmax[q], key);
                            kinv[q] = max(kinv[q], ~key);
                        }
                    }
                }
            }
        }
    }
    if (first) {
        const double r = block_sum(sum, sh_red);
        if (threadIdx.x == 0) part_sum[(size_t)j * gridDim.x + blockIdx.x] = r;
    }
    // a problem that shares its source's candidates shares its extremes
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
#pragma unroll
        for (int r = 0; r < NQ; ++r)
            if (r < q && src[q] == r) {
                kmax[q] = kmax[r];
                kinv[q] = kinv[r];
            }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (q >= n_p || done[q]) continue;
        const unsigned long long a = block_max_u64(kmax[q], sh_red_u);
        const unsigned long long b = block_max_u64(kinv[q], sh_red_u);
        if (threadIdx.x == 0) {
            atomicMax(&minmax[2 * ((size_t)j * n_p + q)], a);
            atomicMax(&minmax[2 * ((size_t)j * n_p + q) + 1], b);
        }
    }
    __syncthreads();
    unsigned int* gh = ghist + ((size_t)j * n_p) * kMaxBins;
    for (int i = threadIdx.x; i < n_p * nb; i += blockDim.x) {
        const int q = i >> bits, b = i & (int)dmask;
        const unsigned c = sh_hist[sh_src[q] * nb + b];  // zero for a decided problem
        if (c) atomicAdd(&gh[(size_t)q * kMaxBins + b], c);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh_last = atomicAdd(&tickets[j], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    for (int q = 0; q < n_p; ++q) {
        if (done[q]) continue;
        SelState* sq = &st[j * n_p + q];
        unsigned long long* mm = &minmax[2 * ((size_t)j * n_p + q)];
        const unsigned long long hi = __ldcg(mm), lo = ~__ldcg(mm + 1);
        if (hi == lo) {
            // every candidate holds the same key (a capped layer's AggL, say):
            // the k-th largest is decided without the remaining digits
            if (threadIdx.x == 0) {
                sq->prefix = hi;
                sq->mask = kAllKeyBits;
                sq->krem = 1;
                if (first) sq->k = kq.k[q];
            }
            for (int i = threadIdx.x; i < nb; i += blockDim.x) gh[(size_t)q * kMaxBins + i] = 0;
        } else {
            select_block(sq, gh + (size_t)q * kMaxBins, shift, bits, first, kq.k[q]);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            mm[0] = 0;
            mm[1] = 0;
        }
    }
    if (threadIdx.x == 0) tickets[j] = 0;
}

// The tail sums fused with the final reduction: every block writes its
// partial count and sum of values strictly above each problem's k-th key;
// the last block of the grid (ticket counter) sums the partials of every
// problem in a fixed order (one warp per problem) and writes mean, PML and
// TVaR.
template <int NQ>
__global__ void __launch_bounds__(kThreads) tail_final_kernel(const double* __restrict__ ylt, int64_t n, int n_layers,
                                                              int n_p, const SelState* __restrict__ st,
                                                              const double* __restrict__ mean_part,
                                                              unsigned long long* __restrict__ part_cnt,
                                                              double* __restrict__ part_sum,
                                                              unsigned int* __restrict__ ticket, double* mean,
                                                              double* pml, double* tvar) {
    __shared__ double sh_red[32];
    __shared__ unsigned long long sh_red_u[32];
    __shared__ bool sh_last;
    const int j = blockIdx.y;
    const int nblk = gridDim.x;
    unsigned long long thr[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) thr[q] = q < n_p ? st[j * n_p + q].prefix : ~0ULL;
    const double* row = ylt + (size_t)j * (size_t)n;
    double s[NQ];
    unsigned long long c[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        s[q] = 0.0;
        c[q] = 0;
    }
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kUnroll; i0 < n;
         i0 += (int64_t)gridDim.x * blockDim.x * kUnroll) {
        double v[kUnroll];
        bool valid[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x + threadIdx.x;
            valid[u] = i < n;
            v[u] = valid[u] ? row[i] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const unsigned long long key = valid[u] ? key_of(v[u]) : 0ULL;  // 0: never above a threshold
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < n_p && key > thr[q]) {
                    s[q] += v[u];
                    c[q] += 1;
                }
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (q >= n_p) break;
        const double rs = block_sum(s[q], sh_red);
        const unsigned long long rc = block_sum_u64(c[q], sh_red_u);
        if (threadIdx.x == 0) {
            const size_t w = ((size_t)j * n_p + q) * nblk + blockIdx.x;
            part_sum[w] = rs;
            part_cnt[w] = rc;
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh_last = atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    for (int i = wib; i < n_layers * n_p; i += kThreads / 32) {
        const int jj = i / n_p, q = i % n_p;
        double m = 0.0, sgt = 0.0;
        unsigned long long cgt = 0;
        for (int b0 = 0; b0 < nblk; b0 += 32 * 8) {
            // eight partials per lane requested at once, then summed in order
            double pm[8], ps[8];
            unsigned long long pc[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int b = b0 + r * 32 + lane;
                const bool ok = b < nblk;
                pm[r] = ok && q == 0 ? __ldcg(mean_part + (size_t)jj * nblk + b) : 0.0;
                ps[r] = ok ? __ldcg(part_sum + (size_t)i * nblk + b) : 0.0;
                pc[r] = ok ? __ldcg(part_cnt + (size_t)i * nblk + b) : 0ULL;
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                m += pm[r];
                sgt += ps[r];
                cgt += pc[r];
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            m += __shfl_xor_sync(0xffffffffu, m, o);
            sgt += __shfl_xor_sync(0xffffffffu, sgt, o);
            cgt += __shfl_xor_sync(0xffffffffu, cgt, o);
        }
        if (lane == 0) {
            if (q == 0 && mean) mean[jj] = m / (double)n;
            const double v = __longlong_as_double((long long)__ldcg(&st[i].prefix));
            const long long k = __ldcg(&st[i].k);
            if (pml) pml[i] = v;
            if (tvar) tvar[i] = (sgt + (double)(k - (long long)cgt) * v) / (double)k;
        }
    }
    if (threadIdx.x == 0) *ticket = 0;
}

// The metric kernels over caller-provided scratch: six fused radix passes,
// then the fused tail and final reduction (seven launches). hist and the
// tickets (contiguous, n_layers + 1 counters after the bins) must be zero.
cudaError_t launch_metric_kernels(const double* ylt, int64_t n, int32_t n_layers, int32_t n_p, const KParams& kq,
                                  int nblk, SelState* st, unsigned int* hist, unsigned long long* minmax,
                                  unsigned int* tickets, double* msum, unsigned long long* tcnt, double* tsum,
                                  double* mean, double* pml, double* tvar, cudaStream_t s) {
    // the probability loops are compiled for 1, 2, 4 or 8 problems per layer
    auto hist_k = n_p <= 1 ? hist_select_kernel<1> : n_p <= 2 ? hist_select_kernel<2>
                : n_p <= 4 ? hist_select_kernel<4> : hist_select_kernel<8>;
    auto tail_k = n_p <= 1 ? tail_final_kernel<1> : n_p <= 2 ? tail_final_kernel<2>
                : n_p <= 4 ? tail_final_kernel<4> : tail_final_kernel<8>;
    cudaError_t err = cudaSuccess;
    for (int i = 0; i < kPasses && !err; ++i) {
        const int bits = pass_bits(i);
        const size_t shm = sizeof(unsigned int) * (size_t)n_p << bits;
        if (shm > 48 * 1024 && (err = cudaFuncSetAttribute(hist_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm)))
            break;
        hist_k<<<dim3(nblk, n_layers), kThreads, shm, s>>>(ylt, n, n_p, st, pass_shift(i), bits, i == 0, kq, hist,
                                                           minmax, msum, tickets);
        err = cudaGetLastError();
    }
    if (err) return err;
    tail_k<<<dim3(nblk, n_layers), kThreads, 0, s>>>(ylt, n, n_layers, n_p, st, msum, tcnt, tsum, tickets + n_layers,
                                                     mean, pml, tvar);
    return cudaGetLastError();
}

int blocks_per_layer(int64_t n, int n_layers) {
    int dev = 0, sms = 148, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    // about 16 values per thread (4 steps of kUnroll)
    int64_t want = (n + (int64_t)kThreads * 16 - 1) / ((int64_t)kThreads * 16);
    // a YLT larger than L2 streams from HBM in every pass, and more blocks
    // keep more of its loads in flight (8 per SM); one that L2 holds is
    // re-read from L2, where each block's fixed cost (clearing, flushing
    // and ticketing its histograms) weighs more (4 per SM)
    const bool streamed = (double)n * (double)n_layers * sizeof(double) > (double)l2;
    const int64_t per_sm = streamed ? 8 : 4;
    int64_t cap = std::max<int64_t>(1, (per_sm * sms + n_layers - 1) / n_layers);
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

int64_t tail_count(double p, int64_t n) {
    if (n <= 0) return 0;
    const double q = (1.0 - p) * (double)n;
    const double r = std::nearbyint(q);
    int64_t k = (std::fabs(q - r) <= 1e-9 * (double)n) ? (int64_t)r : (int64_t)std::ceil(q);
    return std::min<int64_t>(n, std::max<int64_t>(1, k));
}

cudaError_t metrics_run(const double* ylt, int64_t n, int32_t n_layers, const double* probs, int32_t n_p,
                        double* mean, double* pml, double* tvar, cudaStream_t s) {
    const int nblk = blocks_per_layer(n, n_layers);
    const int n_prob = n_layers * n_p;
    // scratch: state, histograms and tickets (zeroed together), partial sums
    const size_t o_st = 0;
    const size_t o_h = align256(o_st + sizeof(SelState) * n_prob);
    // bins, then per problem the candidates' largest key and complement, then
    // the tickets: zeroed together
    const size_t hist_bytes = sizeof(unsigned int) * kMaxBins * (size_t)n_prob +
                              sizeof(unsigned long long) * 2 * (size_t)n_prob + sizeof(unsigned int) * (n_layers + 1);
    const size_t o_ms = align256(o_h + hist_bytes);
    const size_t o_tc = align256(o_ms + sizeof(double) * (size_t)n_layers * nblk);
    const size_t o_ts = align256(o_tc + sizeof(unsigned long long) * (size_t)n_prob * nblk);
    const size_t total = align256(o_ts + sizeof(double) * (size_t)n_prob * nblk);
    char* w = nullptr;
    cudaError_t err = cudaMallocAsync((void**)&w, total, s);
    if (err != cudaSuccess) return err;
    KParams kq = {};
    for (int q = 0; q < n_p; ++q) kq.k[q] = tail_count(probs[q], n);
    auto* hist = (unsigned int*)(w + o_h);
    err = cudaMemsetAsync(hist, 0, hist_bytes, s);
    if (!err)
        err = launch_metric_kernels(ylt, n, n_layers, n_p, kq, nblk, (SelState*)(w + o_st), hist,
                                    (unsigned long long*)(hist + kMaxBins * (size_t)n_prob),
                                    (unsigned int*)((unsigned long long*)(hist + kMaxBins * (size_t)n_prob) +
                                                    2 * (size_t)n_prob),
                                    (double*)(w + o_ms),
                                    (unsigned long long*)(w + o_tc), (double*)(w + o_ts), mean, pml, tvar, s);
    const cudaError_t e2 = cudaFreeAsync(w, s);
    return err ? err : e2;
}

cudaError_t metrics_backward_run(const double* ylt, int64_t n, int32_t n_layers, const double* probs, int32_t n_p,
                                 const double* pml, const double* gmean, const double* gtvar, double* gylt,
                                 cudaStream_t s) {
    const int nblk = blocks_per_layer(n, n_layers);
    const int n_prob = n_layers * n_p;
    const size_t o_g = 0;
    const size_t o_e = align256(o_g + sizeof(unsigned long long) * (size_t)n_prob * nblk);
    const size_t o_wg = align256(o_e + sizeof(unsigned long long) * (size_t)n_prob * nblk);
    const size_t o_we = align256(o_wg + sizeof(double) * n_prob);
    const size_t total = align256(o_we + sizeof(double) * n_prob);
    char* w = nullptr;
    cudaError_t err = cudaMallocAsync((void**)&w, total, s);
    if (err != cudaSuccess) return err;
    KParams kq = {};
    for (int q = 0; q < n_p; ++q) kq.k[q] = tail_count(probs[q], n);
    auto* pg = (unsigned long long*)(w + o_g);
    auto* pe = (unsigned long long*)(w + o_e);
    auto* wg = (double*)(w + o_wg);
    auto* we = (double*)(w + o_we);
    do {
        // the probability loops are compiled for 1, 2, 4 or 8 problems per layer
        auto count_k = n_p <= 1 ? count_kernel<1> : n_p <= 2 ? count_kernel<2>
                     : n_p <= 4 ? count_kernel<4> : count_kernel<8>;
        auto grad_k = n_p <= 1 ? grad_ylt_kernel<1> : n_p <= 2 ? grad_ylt_kernel<2>
                    : n_p <= 4 ? grad_ylt_kernel<4> : grad_ylt_kernel<8>;
        if (gtvar) {
            count_k<<<dim3(nblk, n_layers), kThreads, 0, s>>>(ylt, n, n_p, pml, pg, pe);
            if ((err = cudaGetLastError())) break;
            weights_kernel<<<(n_prob + 127) / 128, 128, 0, s>>>(n_layers, n_p, nblk, kq, pg, pe, wg, we);
            if ((err = cudaGetLastError())) break;
        }
        grad_k<<<dim3(nblk, n_layers), kThreads, 0, s>>>(ylt, n, gtvar ? n_p : 0, pml, gmean, gtvar, wg, we, gylt);
        err = cudaGetLastError();
    } while (0);
    const cudaError_t e2 = cudaFreeAsync(w, s);
    return err ? err : e2;
}

}  // namespace art

// ---------------------------------------------------------------------------
// art_metrics_noalloc: the same kernels over a fixed scratch array that the
// library defines at file scope, for callers that cannot allocate device
// memory (see include/art.h). The array lives in every device's copy of this
// module; host code never dereferences its name, it asks the runtime for the
// device address once per device.
#include <mutex>

namespace art {

static __device__ __align__(256) unsigned char g_metrics_noalloc_scratch[ART_METRICS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device, looked up on
// the first call per device (with that device current) and cached.
cudaError_t noalloc_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_metrics_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = static_cast<unsigned char*>(ptr);
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace art

extern "C" art_status art_metrics_noalloc(const double* ylt_dev, int64_t n_trials, int32_t n_layers,
                                          const double* probs_host, int32_t n_p, double* mean_dev, double* pml_dev,
                                          double* tvar_dev, cudaStream_t stream) {
    using namespace art;
    if (!ylt_dev || n_trials < 1 || n_trials > 0x7fffffffLL || n_layers < 1 || n_layers > 65535 || !probs_host ||
        n_p < 1 || n_p > kMaxProbs)
        return ART_EINVAL;
    for (int q = 0; q < n_p; ++q)
        if (!(probs_host[q] > 0.0 && probs_host[q] < 1.0)) return ART_EINVAL;
    const int nblk = blocks_per_layer(n_trials, n_layers);
    const int n_prob = n_layers * n_p;
    const size_t o_st = 0;
    const size_t o_h = align256(o_st + sizeof(SelState) * n_prob);
    // bins, then per problem the candidates' largest key and complement, then
    // the tickets: zeroed together
    const size_t hist_bytes = sizeof(unsigned int) * kMaxBins * (size_t)n_prob +
                              sizeof(unsigned long long) * 2 * (size_t)n_prob + sizeof(unsigned int) * (n_layers + 1);
    const size_t o_ms = align256(o_h + hist_bytes);
    const size_t o_tc = align256(o_ms + sizeof(double) * (size_t)n_layers * nblk);
    const size_t o_ts = align256(o_tc + sizeof(unsigned long long) * (size_t)n_prob * nblk);
    const size_t total = align256(o_ts + sizeof(double) * (size_t)n_prob * nblk);
    if (total > (size_t)ART_METRICS_NOALLOC_SCRATCH_BYTES) return ART_EINVAL;
    unsigned char* w = nullptr;
    cudaError_t err = noalloc_scratch(&w);
    if (err != cudaSuccess) {
        set_last_error(err);
        return ART_ECUDA;
    }
    KParams kq = {};
    for (int q = 0; q < n_p; ++q) kq.k[q] = tail_count(probs_host[q], n_trials);
    auto* hist = (unsigned int*)(w + o_h);
    // the scratch keeps the previous call's contents: the histograms and the
    // tickets must start at zero
    err = cudaMemsetAsync(hist, 0, hist_bytes, stream);
    if (!err)
        err = launch_metric_kernels(ylt_dev, n_trials, n_layers, n_p, kq, nblk, (SelState*)(w + o_st), hist,
                                    (unsigned long long*)(hist + kMaxBins * (size_t)n_prob),
                                    (unsigned int*)((unsigned long long*)(hist + kMaxBins * (size_t)n_prob) +
                                                    2 * (size_t)n_prob),
                                    (double*)(w + o_ms),
                                    (unsigned long long*)(w + o_tc), (double*)(w + o_ts), mean_dev, pml_dev,
                                    tvar_dev, stream);
    if (err != cudaSuccess) {
        set_last_error(err);
        return ART_ECUDA;
    }
    return ART_OK;
}

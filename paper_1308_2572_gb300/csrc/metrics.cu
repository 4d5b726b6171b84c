// metrics.cu -- expected loss, PML and TVaR from the YLT (Section I names PML
// and TVaR as the risk metrics derived from a YLT; Section II applies
// "financial functions or filters" to the trial losses).
//
// Reading: per layer, with k = ceil((1-p) N) (at least 1), PML_p is the k-th
// largest trial loss and TVaR_p the mean of the k largest.
//
// Exact selection without a sort: trial losses are >= 0, so the FP64 bit
// pattern (sign cleared, which also folds -0 onto +0) orders like the value.
// A most-significant-digit radix select over the 63 key bits narrows, for
// every (layer, probability) problem at once, the prefix of the k-th largest
// key: a first digit of 13 bits (the binary exponent and two leading mantissa
// bits), then digits of 11, 11, 11, 11 and 6 bits. Each pass is one launch:
// its blocks histogram the keys that match the prefix found so far
// (shared-memory histograms with warp-aggregated atomics, flushed to global
// with atomics), and the last block of each layer to finish (a ticket counter
// after a fence; no block waits for another) picks the digit where the count
// from the top crosses the remaining rank. A problem whose candidates all
// hold one key is decided at once.
//
// Only the first two passes read the whole YLT. The first also sums each
// layer for the mean and records its smallest and largest key; its last block
// lays out, per layer, a candidate list as long as the first-digit buckets
// its problems selected (while the lists fit the scratch). The second pass
// copies into that list every key of those buckets other than 0 and the
// layer's largest key -- the two values that repeat most (trials without a
// loss, trials at the aggregate cap), which are only counted -- and sums, in
// a fixed order, the values above each problem's bucket. The remaining
// passes and the tail read the candidate list alone, adding the counted keys
// to the histograms where they match. The tail sums the candidates above the
// k-th largest key of the problem's bucket as integers: they share one binary
// exponent, so their mantissas add exactly and in any order. TVaR is
// (sum_gt + (k - count_gt) PML) / k. A layer whose candidates do not fit
// keeps reading its whole row in every pass, and its tail sums in a fixed
// order. Every sum is deterministic.
#include <algorithm>
#include <cmath>

#include "art_internal.cuh"

namespace art {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 8;        // values per thread whose loads are in flight together
constexpr int kPasses = 6;
constexpr int kBins1 = 8192;      // first digit: key bits 62..50
constexpr int kMaxBins = 2048;    // later digits: 11 bits (the last one 6)
constexpr int kShift1 = 50;
__host__ __device__ constexpr int pass_shift(int i) { return i == 0 ? kShift1 : (i < 5 ? kShift1 - 11 * i : 0); }
__host__ __device__ constexpr int pass_bits(int i) { return i == 0 ? 13 : (i < 5 ? 11 : 6); }
constexpr unsigned long long kAllKeyBits = 0x7fffffffffffffffULL;  // a decided problem's mask
constexpr unsigned long long kMant = (1ULL << 52) - 1;

struct KParams {
    long long k[kMaxProbs];
};

// Selection state of one (layer, probability) problem.
struct SelState {
    unsigned long long prefix;  // key bits found so far (the k-th largest key once decided)
    unsigned long long mask;    // which bits prefix holds
    long long krem;             // rank of the k-th largest among the keys matching prefix
    long long k;
    long long above1;           // keys above the first-digit bucket
    unsigned long long b1;      // the first-digit bucket (key >> 50)
    int first_decided;          // decided in the first pass (a constant layer)
    int pad_;
};

// Per-layer state; every field but need, cand_off and compact starts at zero.
struct LayerState {
    unsigned long long kmax, kinv;         // largest key, complement of the smallest (first pass)
    unsigned long long cnt_zero, cnt_max;  // keys equal to 0 / to kmax (second pass, compacted layers)
    unsigned long long need;               // candidate slots the selected buckets hold (first pass)
    unsigned long long cand_off;           // the layer's candidate list in the scratch
    unsigned int cand_n;                   // candidates written (second pass)
    int compact;                           // later passes read the candidate list
};

__device__ __forceinline__ unsigned long long key_of(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

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

// Histogram add for the lanes with `hit`, warp-aggregated: when every such
// lane has the same digit (losses cluster: a capped layer, zero trials) one
// lane adds them all; otherwise lanes with equal digits add once each.
// Called by the whole warp.
__device__ __forceinline__ void hist_add(unsigned int* h, unsigned dig, bool hit, unsigned lane) {
    const unsigned act = __ballot_sync(0xffffffffu, hit);
    if (!act) return;
    const int first = __ffs(act) - 1;
    const unsigned d0 = __shfl_sync(0xffffffffu, dig, first);
    if (__all_sync(0xffffffffu, !hit || dig == d0)) {
        if (lane == (unsigned)first) atomicAdd(h + d0, __popc(act));
        return;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, hit ? dig : 0xffffffffu);
    if (hit && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(h + dig, __popc(peers));
}

// Block-wide digit pick: the bin of bins[0, nb) (shared memory) where the
// count of keys from the top reaches krem, and the count in the bins above
// it. Valid in every thread on return.
__device__ void pick_digit(const unsigned int* bins, int nb, long long krem, int* bin_out,
                           unsigned long long* above_out) {
    __shared__ unsigned long long sh_scan[kThreads];
    __shared__ int sh_bin;
    __shared__ unsigned long long sh_above;
    const int per = (nb + kThreads - 1) / kThreads;
    // thread i covers descending ranks [i*per, (i+1)*per): bins nb-1-i*per downwards
    unsigned long long local = 0;
    for (int r = 0; r < per; ++r) {
        const int idx = threadIdx.x * per + r;
        if (idx < nb) local += bins[nb - 1 - idx];
    }
    sh_scan[threadIdx.x] = local;
    if (threadIdx.x == 0) {
        sh_bin = -1;
        sh_above = 0;
    }
    __syncthreads();
    for (int o = 1; o < kThreads; o <<= 1) {
        const unsigned long long add = threadIdx.x >= (unsigned)o ? sh_scan[threadIdx.x - o] : 0ULL;
        __syncthreads();
        sh_scan[threadIdx.x] += add;
        __syncthreads();
    }
    const unsigned long long incl = sh_scan[threadIdx.x];
    const unsigned long long excl = incl - local;
    if ((long long)excl < krem && krem <= (long long)incl) {
        unsigned long long run = excl;
        for (int r = 0; r < per; ++r) {
            const int idx = threadIdx.x * per + r;
            if (idx >= nb) break;
            const unsigned c = bins[nb - 1 - idx];
            if ((long long)(run + c) >= krem) {
                sh_bin = nb - 1 - idx;
                sh_above = run;
                break;
            }
            run += c;
        }
    }
    __syncthreads();
    *bin_out = sh_bin < 0 ? 0 : sh_bin;  // -1 is unreachable when the counts are consistent
    *above_out = sh_above;
    __syncthreads();
}

// Pass 1 over every value: first-digit histogram (one per layer, shared by
// its problems), the layer's sum for the mean (two FP64 accumulators, fixed
// assignment), its smallest and largest key. The last block of a layer picks
// its problems' first digits; the last layer to be picked lays out the
// candidate lists (greedily, in layer order, while they fit the budget).
__global__ void __launch_bounds__(kThreads) first_pass_kernel(const double* __restrict__ ylt, int64_t n, int n_p,
                                                              const KParams kq, SelState* __restrict__ st,
                                                              LayerState* __restrict__ ls,
                                                              unsigned int* __restrict__ hist1,
                                                              double* __restrict__ part_mean,
                                                              unsigned int* __restrict__ tickets,
                                                              unsigned long long cand_budget) {
    extern __shared__ unsigned int sh_hist[];  // [kBins1]
    __shared__ double sh_red[32];
    __shared__ unsigned long long sh_red_u[32];
    __shared__ bool sh_last;
    __shared__ unsigned long long sh_need[kThreads];
    const int j = blockIdx.y;
    const int n_layers = gridDim.y;
    const unsigned lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < kBins1; i += blockDim.x) sh_hist[i] = 0;
    __syncthreads();
    const double* row = ylt + (size_t)j * (size_t)n;
    double s0 = 0.0, s1 = 0.0;
    unsigned long long kmax = 0, kinv = 0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kUnroll; i0 < n;
         i0 += (int64_t)gridDim.x * blockDim.x * kUnroll) {
        double v[kUnroll];
        bool valid[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x + threadIdx.x;
            valid[u] = i < n;
            v[u] = valid[u] ? __ldcs(row + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if (u & 1) s1 += v[u];
            else s0 += v[u];
            const unsigned long long key = key_of(v[u]);
            hist_add(sh_hist, (unsigned)(key >> kShift1), valid[u], lane);
            if (valid[u]) {
                kmax = max(kmax, key);
                kinv = max(kinv, ~key);
            }
        }
    }
    const double r = block_sum(s0 + s1, sh_red);
    if (threadIdx.x == 0) part_mean[(size_t)j * gridDim.x + blockIdx.x] = r;
    const unsigned long long a = block_max_u64(kmax, sh_red_u);
    const unsigned long long b = block_max_u64(kinv, sh_red_u);
    if (threadIdx.x == 0) {
        atomicMax(&ls[j].kmax, a);
        atomicMax(&ls[j].kinv, b);
    }
    __syncthreads();
    unsigned int* gh = hist1 + (size_t)j * kBins1;
    for (int i = threadIdx.x; i < kBins1; i += blockDim.x) {
        const unsigned c = sh_hist[i];
        if (c) atomicAdd(&gh[i], c);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh_last = atomicAdd(&tickets[j], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    // the layer's complete histogram
    for (int i = threadIdx.x; i < kBins1; i += blockDim.x) sh_hist[i] = __ldcg(&gh[i]);
    const unsigned long long hi = __ldcg(&ls[j].kmax), lo = ~__ldcg(&ls[j].kinv);
    __syncthreads();
    for (int q = 0; q < n_p; ++q) {
        SelState* sq = &st[j * n_p + q];
        if (hi == lo) {
            // a constant layer: every problem is decided by its one key
            if (threadIdx.x == 0)
                *sq = SelState{hi, kAllKeyBits, 1, kq.k[q], 0, hi >> kShift1, 1, 0};
        } else {
            int bin;
            unsigned long long above;
            pick_digit(sh_hist, kBins1, kq.k[q], &bin, &above);
            if (threadIdx.x == 0)
                *sq = SelState{(unsigned long long)bin << kShift1, (unsigned long long)(kBins1 - 1) << kShift1,
                               kq.k[q] - (long long)above, kq.k[q], (long long)above, (unsigned long long)bin, 0, 0};
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // candidate slots: the keys of the distinct buckets the problems selected
        unsigned long long need = 0;
        if (hi != lo) {
            for (int q = 0; q < n_p; ++q) {
                const unsigned long long bq = st[j * n_p + q].b1;
                bool seen = false;
                for (int r = 0; r < q; ++r) seen = seen || st[j * n_p + r].b1 == bq;
                if (!seen) need += sh_hist[bq];
            }
        }
        ls[j].need = need;
        tickets[j] = 0;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh_last = atomicAdd(&tickets[n_layers], 1u) == (unsigned)n_layers - 1;
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    // the last layer picked: candidate lists in layer order while they fit
    unsigned long long run = 0;
    for (int c0 = 0; c0 < n_layers; c0 += kThreads) {
        const int jj = c0 + threadIdx.x;
        sh_need[threadIdx.x] = jj < n_layers ? __ldcg(&ls[jj].need) : 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int t = 0; t < kThreads && c0 + t < n_layers; ++t) {
                const unsigned long long nd = sh_need[t];
                const bool fits = run + nd <= cand_budget;
                ls[c0 + t].compact = fits ? 1 : 0;
                ls[c0 + t].cand_off = fits ? run : 0;
                if (fits) run += nd;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) tickets[n_layers] = 0;
}

// Passes 2-6. Each block histograms the keys matching each problem's prefix
// (problems with the same prefix share the histogram of the first of them),
// from the layer's whole row in pass 2 and in every pass of a layer without
// a candidate list, else from the candidate list. Pass 2 also writes the
// candidate lists (keys of the selected first-digit buckets other than 0 and
// the layer's largest key, which it counts), and the per-block sums of the
// values above each problem's bucket. The last block of a layer picks the
// digits; the counted keys enter its histograms and extremes when they match.
template <int NQ>
__global__ void __launch_bounds__(kThreads) pass_kernel(const double* __restrict__ ylt, int64_t n, int n_p,
                                                        SelState* __restrict__ st, LayerState* __restrict__ ls,
                                                        unsigned long long* __restrict__ cand, int shift, int bits,
                                                        bool second, unsigned int* __restrict__ ghist,
                                                        unsigned long long* __restrict__ minmax,
                                                        double* __restrict__ part_above,
                                                        unsigned int* __restrict__ tickets) {
    extern __shared__ unsigned int sh_hist[];  // [n_p][1 << bits]
    __shared__ double sh_red[32];
    __shared__ unsigned long long sh_red_u[32];
    __shared__ bool sh_last;
    __shared__ int sh_src[kMaxProbs];
    const int nb = 1 << bits;
    const int j = blockIdx.y;
    const unsigned lane = threadIdx.x & 31;
    unsigned long long pre[NQ], msk[NQ], b1[NQ];
    bool done[NQ];
    bool all_done = true;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        pre[q] = q < n_p ? st[j * n_p + q].prefix : 1ULL;  // unused slots never match
        msk[q] = q < n_p ? st[j * n_p + q].mask : 0ULL;
        b1[q] = q < n_p ? st[j * n_p + q].b1 : 0ULL;
        done[q] = q >= n_p || msk[q] == kAllKeyBits;
        all_done = all_done && done[q];
    }
    if (all_done) return;  // the same for every block of the layer: no ticket is taken
    const bool compact = ls[j].compact != 0;
    const unsigned long long kmax_l = ls[j].kmax;
    const bool from_row = second || !compact;
    const double* src_vals = from_row ? ylt + (size_t)j * (size_t)n
                                      : reinterpret_cast<const double*>(cand + ls[j].cand_off);
    const int64_t len = from_row ? n : (int64_t)min((unsigned long long)ls[j].cand_n, ls[j].need);
    const bool writing = second && compact;  // pass 2 writes the layer's candidate list
    unsigned long long* my_cand = cand + ls[j].cand_off;
    const unsigned long long cap = ls[j].need;
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
    unsigned long long kmx[NQ], kiv[NQ];
    double sab[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        kmx[q] = 0;
        kiv[q] = 0;
        sab[q] = 0.0;
    }
    unsigned long long czero = 0, cmax = 0;
    __syncthreads();
    const unsigned dmask = (unsigned)nb - 1u;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kUnroll; i0 < len;
         i0 += (int64_t)gridDim.x * blockDim.x * kUnroll) {
        double v[kUnroll];
        bool valid[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x + threadIdx.x;
            valid[u] = i < len;
            v[u] = valid[u] ? __ldcs(src_vals + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const unsigned long long key = key_of(v[u]);
            const unsigned dig = (unsigned)(key >> shift) & dmask;
            bool any = false;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                if (q < n_p && !done[q] && src[q] == q) {  // the same for the whole block
                    const bool hit = valid[u] && (key & msk[q]) == pre[q];
                    any = any || hit;
                    // after the first digits few warps hold a candidate at all
                    if (__any_sync(0xffffffffu, hit)) {
                        hist_add(sh_hist + q * nb, dig, hit, lane);
                        if (hit) {
                            kmx[q] = max(kmx[q], key);
                            kiv[q] = max(kiv[q], ~key);
                        }
                    }
                }
            }
            if (writing) {
                czero += (valid[u] && key == 0ULL) ? 1 : 0;
                cmax += (valid[u] && key == kmax_l) ? 1 : 0;
                const bool c = any && key != 0ULL && key != kmax_l;
                const unsigned m = __ballot_sync(0xffffffffu, c);
                if (m) {
                    const int leader = __ffs(m) - 1;
                    unsigned int base = 0;
                    if (lane == (unsigned)leader) base = atomicAdd(&ls[j].cand_n, (unsigned)__popc(m));
                    base = __shfl_sync(0xffffffffu, base, leader);
                    const unsigned long long slot = (unsigned long long)base + __popc(m & lt_mask);
                    if (c && slot < cap) my_cand[slot] = key;
                }
                // values above each problem's first-digit bucket, for TVaR
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    if (q < n_p && !done[q]) {
                        const bool up = valid[u] && (key >> kShift1) > b1[q];
                        if (__any_sync(0xffffffffu, up) && up) sab[q] += v[u];
                    }
                }
            }
        }
    }
    if (writing) {
        const unsigned long long z = block_sum_u64(czero, sh_red_u);
        const unsigned long long m = block_sum_u64(cmax, sh_red_u);
        if (threadIdx.x == 0) {
            if (z) atomicAdd(&ls[j].cnt_zero, z);
            if (m) atomicAdd(&ls[j].cnt_max, m);
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if (q >= n_p || done[q]) continue;
            const double s = block_sum(sab[q], sh_red);
            if (threadIdx.x == 0) part_above[((size_t)j * n_p + q) * gridDim.x + blockIdx.x] = s;
        }
    }
    // a problem that shares its source's candidates shares its extremes
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
#pragma unroll
        for (int r = 0; r < NQ; ++r)
            if (r < q && src[q] == r) {
                kmx[q] = kmx[r];
                kiv[q] = kiv[r];
            }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (q >= n_p || done[q]) continue;
        const unsigned long long a = block_max_u64(kmx[q], sh_red_u);
        const unsigned long long b = block_max_u64(kiv[q], sh_red_u);
        if (threadIdx.x == 0) {
            if (a) atomicMax(&minmax[2 * ((size_t)j * n_p + q)], a);
            if (b) atomicMax(&minmax[2 * ((size_t)j * n_p + q) + 1], b);
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
    // keys counted instead of listed take part from pass 3 on, where they match
    const bool virt = !second && compact;
    const unsigned long long cz = virt ? __ldcg(&ls[j].cnt_zero) : 0ULL;
    const unsigned long long cm = virt ? __ldcg(&ls[j].cnt_max) : 0ULL;
    for (int q = 0; q < n_p; ++q) {
        if (done[q]) continue;
        SelState* sq = &st[j * n_p + q];
        unsigned long long* mm = &minmax[2 * ((size_t)j * n_p + q)];
        unsigned long long hi = __ldcg(mm), inv = __ldcg(mm + 1);  // inv == 0: no listed candidate
        const bool max_in = cm && (kmax_l & msk[q]) == pre[q];
        const bool zero_in = cz && pre[q] == 0ULL;
        if (max_in) {
            hi = max(hi, kmax_l);
            inv = max(inv, ~kmax_l);
        }
        if (zero_in) inv = ~0ULL;  // the smallest key is 0
        const unsigned long long lo = ~inv;
        unsigned int* gq = gh + (size_t)q * kMaxBins;
        if (hi == lo) {
            // every candidate holds the same key: the k-th largest is decided
            if (threadIdx.x == 0) {
                sq->prefix = hi;
                sq->mask = kAllKeyBits;
                sq->krem = 1;
            }
        } else {
            for (int i = threadIdx.x; i < nb; i += blockDim.x) sh_hist[i] = __ldcg(gq + i);
            __syncthreads();
            if (threadIdx.x == 0) {
                if (max_in) sh_hist[(kmax_l >> shift) & dmask] += (unsigned)cm;
                if (zero_in) sh_hist[0] += (unsigned)cz;
            }
            __syncthreads();
            int bin;
            unsigned long long above;
            pick_digit(sh_hist, nb, sq->krem, &bin, &above);
            if (threadIdx.x == 0) {
                sq->prefix = pre[q] | (unsigned long long)bin << shift;
                sq->mask = msk[q] | (unsigned long long)dmask << shift;
                sq->krem -= (long long)above;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += blockDim.x) gq[i] = 0;
        if (threadIdx.x == 0) {
            mm[0] = 0;
            mm[1] = 0;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) tickets[j] = 0;
}

// Exact sum of keys that share one binary exponent e (the bucket's): their
// mantissas (with the implicit bit when e > 0) as integers, split at bit 32
// so that neither half overflows for 2^31 values.
struct MantSum {
    unsigned long long hi, lo, cnt;
};

__device__ __forceinline__ unsigned long long mant_of(unsigned long long key) {
    const unsigned long long e = key >> 52;
    return (key & kMant) | (e ? (1ULL << 52) : 0ULL);
}

// Value of an exact mantissa sum for exponent field e: one rounding.
__device__ __forceinline__ double mant_value(unsigned long long hi, unsigned long long lo, unsigned long long e) {
    const unsigned long long th = hi + (lo >> 32), tl = lo & 0xffffffffULL;
    const double t = fma((double)th, 4294967296.0, (double)tl);
    return scalbn(t, (int)(e ? e : 1) - 1075);
}

// The tail, fused with the final reduction. Layers with candidate lists: the
// candidates of each problem's bucket above its k-th largest key, summed as
// integers (atomics on exact integers: any order gives the same bits).
// Layers without: every value above the k-th largest key, summed in FP64 per
// block in a fixed order (skipped when the k-th largest is the layer's
// largest key). The last block of the grid reduces every problem in a fixed
// order (one warp per problem) and writes mean, PML and TVaR.
template <int NQ>
__global__ void __launch_bounds__(kThreads) tail_kernel(const double* __restrict__ ylt, int64_t n, int n_p,
                                                        const SelState* __restrict__ st,
                                                        const LayerState* __restrict__ ls,
                                                        const unsigned long long* __restrict__ cand,
                                                        const double* __restrict__ part_mean,
                                                        const double* __restrict__ part_above,
                                                        double* __restrict__ part_sum,
                                                        unsigned long long* __restrict__ part_cnt,
                                                        unsigned long long* __restrict__ int_acc,
                                                        unsigned int* __restrict__ ticket, double* mean, double* pml,
                                                        double* tvar, double* sum_out) {
    __shared__ double sh_red[32];
    __shared__ unsigned long long sh_red_u[32];
    __shared__ bool sh_last;
    const int j = blockIdx.y;
    const int n_layers = gridDim.y;
    const int nblk = gridDim.x;
    const bool compact = ls[j].compact != 0;
    const unsigned long long kmax_l = ls[j].kmax;
    unsigned long long thr[NQ], b1[NQ];
    bool live[NQ];
    bool any_live = false;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        thr[q] = q < n_p ? st[j * n_p + q].prefix : ~0ULL;
        b1[q] = q < n_p ? st[j * n_p + q].b1 : 0ULL;
        // nothing lies above the k-th largest key when it is the layer's largest
        live[q] = q < n_p && !st[j * n_p + q].first_decided && (compact || thr[q] != kmax_l);
        any_live = any_live || live[q];
    }
    if (compact) {
        const unsigned long long* c = cand + ls[j].cand_off;
        const int64_t len = any_live ? (int64_t)min((unsigned long long)ls[j].cand_n, ls[j].need) : 0;
        unsigned long long mh[NQ], ml[NQ], mc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) mh[q] = ml[q] = mc[q] = 0;
        for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kUnroll; i0 < len;
             i0 += (int64_t)gridDim.x * blockDim.x * kUnroll) {
            unsigned long long kv[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int64_t i = i0 + (int64_t)u * blockDim.x + threadIdx.x;
                kv[u] = i < len ? __ldcs(c + i) : 0ULL;  // 0: never above a k-th largest key
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const unsigned long long m = mant_of(kv[u]);
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    if (live[q] && (kv[u] >> kShift1) == b1[q] && kv[u] > thr[q]) {
                        mh[q] += m >> 32;
                        ml[q] += m & 0xffffffffULL;
                        mc[q] += 1;
                    }
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if (!live[q]) continue;
            const unsigned long long a = block_sum_u64(mh[q], sh_red_u);
            const unsigned long long b = block_sum_u64(ml[q], sh_red_u);
            const unsigned long long cc = block_sum_u64(mc[q], sh_red_u);
            if (threadIdx.x == 0 && cc) {
                unsigned long long* acc = int_acc + 3 * ((size_t)j * n_p + q);
                atomicAdd(acc, a);
                atomicAdd(acc + 1, b);
                atomicAdd(acc + 2, cc);
            }
        }
    } else {
        const double* row = ylt + (size_t)j * (size_t)n;
        const int64_t len = any_live ? n : 0;
        double s[NQ];
        unsigned long long cnt[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            s[q] = 0.0;
            cnt[q] = 0;
        }
        for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kUnroll; i0 < len;
             i0 += (int64_t)gridDim.x * blockDim.x * kUnroll) {
            double v[kUnroll];
            bool valid[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int64_t i = i0 + (int64_t)u * blockDim.x + threadIdx.x;
                valid[u] = i < len;
                v[u] = valid[u] ? __ldcs(row + i) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const unsigned long long key = valid[u] ? key_of(v[u]) : 0ULL;  // 0: never above
#pragma unroll
                for (int q = 0; q < NQ; ++q)
                    if (live[q] && key > thr[q]) {
                        s[q] += v[u];
                        cnt[q] += 1;
                    }
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if (q >= n_p) break;
            const double rs = block_sum(s[q], sh_red);
            const unsigned long long rc = block_sum_u64(cnt[q], sh_red_u);
            if (threadIdx.x == 0) {
                const size_t w = ((size_t)j * n_p + q) * nblk + blockIdx.x;
                part_sum[w] = rs;
                part_cnt[w] = rc;
            }
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
        const SelState sq = st[i];
        const bool cmp = __ldcg(&ls[jj].compact) != 0;
        double m = 0.0, s = 0.0;
        unsigned long long c = 0;
        for (int b0 = 0; b0 < nblk; b0 += 32 * 8) {
            // eight partials per lane requested at once, then summed in order
            double pm[8], ps[8];
            unsigned long long pc[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int b = b0 + r * 32 + lane;
                const bool ok = b < nblk;
                pm[r] = ok && q == 0 ? __ldcg(part_mean + (size_t)jj * nblk + b) : 0.0;
                ps[r] = ok ? __ldcg((cmp ? part_above : part_sum) + (size_t)i * nblk + b) : 0.0;
                pc[r] = ok && !cmp ? __ldcg(part_cnt + (size_t)i * nblk + b) : 0ULL;
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                m += pm[r];
                s += ps[r];
                c += pc[r];
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            m += __shfl_xor_sync(0xffffffffu, m, o);
            s += __shfl_xor_sync(0xffffffffu, s, o);
            c += __shfl_xor_sync(0xffffffffu, c, o);
        }
        if (lane == 0) {
            if (q == 0 && mean) mean[jj] = m / (double)n;
            if (q == 0 && sum_out) sum_out[jj] = m;
            const double v = __longlong_as_double((long long)sq.prefix);
            if (sq.first_decided) {
                s = 0.0;  // a constant layer: nothing above its one key
                c = 0;
            } else if (cmp) {
                // above the bucket (pass 2) plus the bucket's keys above the
                // k-th largest: the listed ones and the counted largest key
                const unsigned long long* acc = int_acc + 3 * (size_t)i;
                unsigned long long mh = __ldcg(acc), ml = __ldcg(acc + 1), mc = __ldcg(acc + 2);
                const unsigned long long kmx = __ldcg(&ls[jj].kmax), cm = __ldcg(&ls[jj].cnt_max);
                if (cm && (kmx >> kShift1) == sq.b1 && kmx > sq.prefix) {
                    const unsigned long long mk = mant_of(kmx);
                    mh += cm * (mk >> 32);
                    ml += cm * (mk & 0xffffffffULL);
                    mc += cm;
                }
                if (mc) s += mant_value(mh, ml, sq.b1 >> 2);
                c = (unsigned long long)sq.above1 + mc;
            }
            if (pml) pml[i] = v;
            if (tvar) tvar[i] = (s + (double)(sq.k - (long long)c) * v) / (double)sq.k;
        }
    }
    if (threadIdx.x == 0) *ticket = 0;
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

int blocks_per_layer(int64_t n, int n_layers) {
    int dev = 0, sms = 148, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    // about 32 values per thread (4 steps of kUnroll)
    int64_t want = (n + (int64_t)kThreads * 32 - 1) / ((int64_t)kThreads * 32);
    // a YLT larger than L2 streams from HBM in the two full passes, and more
    // blocks keep more of its loads in flight (8 per SM); one that L2 holds
    // is re-read from L2, where each block's fixed cost (clearing, flushing
    // and ticketing its histograms) weighs more (4 per SM)
    const bool streamed = (double)n * (double)n_layers * sizeof(double) > (double)l2;
    const int64_t per_sm = streamed ? 8 : 4;
    int64_t cap = std::max<int64_t>(1, (per_sm * sms + n_layers - 1) / n_layers);
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Scratch of one metrics call, in bytes from its start. The region [zero,
// zero + zero_bytes) must be zero when the call starts; the rest is written
// before it is read. The candidate lists take cand_slots 8-byte keys.
struct MetricsLayout {
    size_t st, ls, hist1, hist, minmax, tickets, above, iacc, pmean, psum, pcnt, cand;
    size_t zero, zero_bytes, total;
};

MetricsLayout metrics_layout(int64_t n, int32_t n_layers, int32_t n_p, int nblk, uint64_t cand_slots) {
    (void)n;
    const size_t L = (size_t)n_layers, np = (size_t)n_layers * n_p, nb = (size_t)nblk;
    MetricsLayout m{};
    m.st = 0;
    m.ls = align256(m.st + sizeof(SelState) * np);
    m.hist1 = align256(m.ls + sizeof(LayerState) * L);
    m.hist = align256(m.hist1 + sizeof(unsigned int) * kBins1 * L);
    m.minmax = align256(m.hist + sizeof(unsigned int) * kMaxBins * np);
    m.tickets = align256(m.minmax + sizeof(unsigned long long) * 2 * np);
    m.above = align256(m.tickets + sizeof(unsigned int) * (L + 2));
    m.iacc = align256(m.above + sizeof(double) * np * nb);
    m.pmean = align256(m.iacc + sizeof(unsigned long long) * 3 * np);
    m.zero = m.ls;
    m.zero_bytes = m.pmean - m.ls;
    m.psum = align256(m.pmean + sizeof(double) * L * nb);
    m.pcnt = align256(m.psum + sizeof(double) * np * nb);
    m.cand = align256(m.pcnt + sizeof(unsigned long long) * np * nb);
    m.total = align256(m.cand + sizeof(unsigned long long) * (size_t)cand_slots);
    return m;
}

// Candidate slots the allocating path reserves: an eighth of the YLT (the
// buckets the problems select hold a few percent of a layer's trials once 0
// and the layer's largest key are left out), at least 65,536, at most the
// whole YLT.
uint64_t default_cand_slots(int64_t n, int32_t n_layers) {
    const uint64_t all = (uint64_t)n * (uint64_t)n_layers;
    return std::min<uint64_t>(all, std::max<uint64_t>(all / 8, 65536));
}

// The metric kernels over a caller's scratch laid out by metrics_layout:
// clear, pass 1, passes 2-6, tail with the final reduction (eight steps on
// the stream, seven of them launches).
cudaError_t launch_metric_kernels(const double* ylt, int64_t n, int32_t n_layers, int32_t n_p, const KParams& kq,
                                  int nblk, char* w, const MetricsLayout& m, uint64_t cand_slots, double* mean,
                                  double* pml, double* tvar, double* sum_out, cudaStream_t s) {
    auto* st = (SelState*)(w + m.st);
    auto* ls = (LayerState*)(w + m.ls);
    auto* hist1 = (unsigned int*)(w + m.hist1);
    auto* hist = (unsigned int*)(w + m.hist);
    auto* minmax = (unsigned long long*)(w + m.minmax);
    auto* tickets = (unsigned int*)(w + m.tickets);
    auto* above = (double*)(w + m.above);
    auto* iacc = (unsigned long long*)(w + m.iacc);
    auto* pmean = (double*)(w + m.pmean);
    auto* psum = (double*)(w + m.psum);
    auto* pcnt = (unsigned long long*)(w + m.pcnt);
    auto* cand = (unsigned long long*)(w + m.cand);
    cudaError_t err = cudaMemsetAsync(w + m.zero, 0, m.zero_bytes, s);
    if (err) return err;
    const dim3 grid(nblk, n_layers);
    first_pass_kernel<<<grid, kThreads, sizeof(unsigned int) * kBins1, s>>>(ylt, n, n_p, kq, st, ls, hist1, pmean,
                                                                            tickets, cand_slots);
    if ((err = cudaGetLastError())) return err;
    // the probability loops are compiled for 1, 2, 4 or 8 problems per layer
    auto pass_k = n_p <= 1 ? pass_kernel<1> : n_p <= 2 ? pass_kernel<2> : n_p <= 4 ? pass_kernel<4> : pass_kernel<8>;
    auto tail_k = n_p <= 1 ? tail_kernel<1> : n_p <= 2 ? tail_kernel<2> : n_p <= 4 ? tail_kernel<4> : tail_kernel<8>;
    for (int i = 1; i < kPasses; ++i) {
        const int bits = pass_bits(i);
        const size_t shm = sizeof(unsigned int) * (size_t)n_p << bits;
        if (shm > 48 * 1024 &&
            (err = cudaFuncSetAttribute(pass_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm)))
            return err;
        pass_k<<<grid, kThreads, shm, s>>>(ylt, n, n_p, st, ls, cand, pass_shift(i), bits, i == 1, hist, minmax,
                                           above, tickets);
        if ((err = cudaGetLastError())) return err;
    }
    tail_k<<<grid, kThreads, 0, s>>>(ylt, n, n_p, st, ls, cand, pmean, above, psum, pcnt, iacc,
                                     tickets + n_layers + 1, mean, pml, tvar, sum_out);
    return cudaGetLastError();
}

}  // namespace

int64_t tail_count(double p, int64_t n) {
    if (n <= 0) return 0;
    const double q = (1.0 - p) * (double)n;
    const double r = std::nearbyint(q);
    int64_t k = (std::fabs(q - r) <= 1e-9 * (double)n) ? (int64_t)r : (int64_t)std::ceil(q);
    return std::min<int64_t>(n, std::max<int64_t>(1, k));
}

cudaError_t metrics_run_k(const double* ylt, int64_t n, int32_t n_layers, const int64_t* k, int32_t n_p,
                          double* mean, double* pml, double* tvar, double* sum_out, cudaStream_t s) {
    const int nblk = blocks_per_layer(n, n_layers);
    const uint64_t slots = default_cand_slots(n, n_layers);
    const MetricsLayout m = metrics_layout(n, n_layers, n_p, nblk, slots);
    char* w = nullptr;
    cudaError_t err = cudaMallocAsync((void**)&w, m.total, s);
    if (err != cudaSuccess) return err;
    KParams kq = {};
    for (int q = 0; q < n_p; ++q) kq.k[q] = std::min<int64_t>(n, std::max<int64_t>(1, k[q]));
    err = launch_metric_kernels(ylt, n, n_layers, n_p, kq, nblk, w, m, slots, mean, pml, tvar, sum_out, s);
    const cudaError_t e2 = cudaFreeAsync(w, s);
    return err ? err : e2;
}

cudaError_t metrics_run(const double* ylt, int64_t n, int32_t n_layers, const double* probs, int32_t n_p,
                        double* mean, double* pml, double* tvar, cudaStream_t s) {
    int64_t k[kMaxProbs];
    for (int q = 0; q < n_p; ++q) k[q] = tail_count(probs[q], n);
    return metrics_run_k(ylt, n, n_layers, k, n_p, mean, pml, tvar, nullptr, s);
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
// device address of the current device's copy.
#include <mutex>

namespace art {

static __device__ __align__(256) unsigned char g_metrics_noalloc_scratch[ART_METRICS_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;

struct NoAllocAddr {
    unsigned char* addr = nullptr;
    unsigned long long ctx_id = 0;  // the context the address belongs to
};
NoAllocAddr g_noalloc[kNoAllocMaxDevices];

// Id of the current device's context (unique over the process's life, so a
// context recreated after cudaDeviceReset gets a new one); 0 if the driver
// cannot tell. Taken from the driver through the runtime's entry-point
// lookup, without linking the driver library.
unsigned long long current_context_id() {
    typedef int (*GetCurrent)(void**);
    typedef int (*GetId)(void*, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of the scratch array on the current device: looked up with
// the device current on the first call, and again whenever the device's
// context has changed since (cudaDeviceReset, or a reset of the primary
// context by another framework, recreates the module and its array), or
// whenever the context cannot be identified.
cudaError_t noalloc_scratch(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocAddr& a = g_noalloc[dev];
    const unsigned long long ctx = current_context_id();
    if (a.addr && ctx != 0 && a.ctx_id == ctx) {
        *out = a.addr;
        return cudaSuccess;
    }
    // the lookup makes the device's primary context current if it was not
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_metrics_noalloc_scratch);
    if (e != cudaSuccess) return e;
    a.addr = static_cast<unsigned char*>(ptr);
    a.ctx_id = current_context_id();
    *out = a.addr;
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
    // the fixed part must fit; what is left holds candidate lists (layers
    // whose lists do not fit read their whole row in every pass instead)
    const MetricsLayout fixed = metrics_layout(n_trials, n_layers, n_p, nblk, 0);
    if (fixed.total > (size_t)ART_METRICS_NOALLOC_SCRATCH_BYTES) return ART_EINVAL;
    const uint64_t slots = std::min<uint64_t>(((size_t)ART_METRICS_NOALLOC_SCRATCH_BYTES - fixed.total) / 8,
                                              default_cand_slots(n_trials, n_layers));
    const MetricsLayout m = metrics_layout(n_trials, n_layers, n_p, nblk, slots);
    if (m.total > (size_t)ART_METRICS_NOALLOC_SCRATCH_BYTES) return ART_EINVAL;
    unsigned char* w = nullptr;
    cudaError_t err = noalloc_scratch(&w);
    if (err != cudaSuccess) {
        set_last_error(err);
        return ART_ECUDA;
    }
    KParams kq = {};
    for (int q = 0; q < n_p; ++q) kq.k[q] = tail_count(probs_host[q], n_trials);
    // the scratch keeps the previous call's contents: the launcher clears
    // what must start at zero
    err = launch_metric_kernels(ylt_dev, n_trials, n_layers, n_p, kq, nblk, reinterpret_cast<char*>(w), m, slots,
                                mean_dev, pml_dev, tvar_dev, nullptr, stream);
    if (err != cudaSuccess) {
        set_last_error(err);
        return ART_ECUDA;
    }
    return ART_OK;
}

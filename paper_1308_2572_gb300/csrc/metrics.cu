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
// its blocks histogram the keys that match the prefix found so far, and the
// last block of each layer to finish (a ticket counter after a fence; no
// block waits for another) picks the digit where the count from the top
// crosses the remaining rank. A problem whose candidates all hold one key is
// decided at once.
//
// Only the first two passes read the whole YLT. Pass 1 histograms the first
// digit and finds each layer's smallest and largest key (zeros are counted in
// registers). Its last blocks lay out, per layer and in layer order while
// they fit the scratch, a candidate list: every key at or above the lowest
// first-digit bucket the layer's problems selected, or, when that does not
// fit, the keys of the selected buckets only. Pass 2 sums each layer for the
// mean and writes the lists, leaving out 0 and the layer's largest key
// (trials without a loss and trials at the aggregate cap, the values that
// repeat most), which it only counts. The remaining passes read the lists
// (the counted keys enter a histogram where they match the prefix). The tail
// sums, per problem, the keys above the k-th largest key: from a list of
// every key above the lowest bucket (plus the counted largest keys when they
// lie above it), else from the row. TVaR = (sum_gt + (k - count_gt) PML) / k.
// A layer without a list histograms its second digit in pass 2 and reads its
// whole row in every later pass.
//
// Every sum is an integer: a value's 53-bit mantissa, shifted to its place
// in a 128-bit fixed-point number whose unit is 2^-96 of the layer's largest
// binary power, added with a carry (bits below the unit are dropped: each
// sum holds the layer's largest loss, so that is at most 2^-96 N of it).
// Integer additions give the same bits in any order, so blocks add their
// sums with atomics, and the streaming passes use no FP64 arithmetic (of
// which this GPU has little). One conversion to FP64 (two roundings) ends
// each sum.
#include <algorithm>
#include <cmath>

#include "art_internal.cuh"

namespace art {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 8;        // values per thread whose loads are in flight together
constexpr int kPasses = 6;        // digits of the radix select
constexpr int kBins1 = 8192;      // first digit: key bits 62..50
constexpr int kMaxBins = 2048;    // later digits: 11 bits (the last one 6)
constexpr int kShift1 = 50;
__host__ __device__ constexpr int pass_shift(int i) { return i == 0 ? kShift1 : (i < 5 ? kShift1 - 11 * i : 0); }
__host__ __device__ constexpr int pass_bits(int i) { return i == 0 ? 13 : (i < 5 ? 11 : 6); }
constexpr unsigned long long kAllKeyBits = 0x7fffffffffffffffULL;  // a decided problem's mask

struct KParams {
    long long k[kMaxProbs];
};

// Selection state of one (layer, probability) problem.
struct SelState {
    unsigned long long prefix;  // key bits found so far (the k-th largest key once decided)
    unsigned long long mask;    // which bits prefix holds
    long long krem;             // rank of the k-th largest among the keys matching prefix
    long long k;
};

// Per-layer state; every field but need, cand_off, compact and stage starts
// at zero.
struct LayerState {
    unsigned long long kmax, kinv;         // largest key, complement of the smallest (pass 1)
    unsigned long long cnt_zero, cnt_max;  // keys equal to 0 / to kmax (pass 1)
    unsigned long long need;               // list slots (pass 1): keys at or above the lowest bucket,
    unsigned long long need_sel;           //   or keys of the selected buckets only
    unsigned long long lo_bucket;          // the lowest selected bucket (key >> 50)
    unsigned long long cand_off;           // the layer's list in the scratch
    unsigned int cand_n;                   // keys listed (pass 2)
    int compact;                           // kListAll, kListSelected or kListNone
    int stage;                             // digits picked so far (kPasses: every problem decided)
};

// What a layer's list holds: every key at or above its lowest selected
// first-digit bucket (the selection and the tail read the list), the keys
// of its selected buckets only (the selection reads the list, the tail the
// row), or nothing (every pass reads the row).
enum { kListNone = 0, kListAll = 1, kListSelected = 2 };

__device__ __forceinline__ unsigned long long key_of(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

// The key of p[i] read as a 64-bit integer (streaming: each value is read
// once per pass), so that no FP64 instruction touches it.
__device__ __forceinline__ unsigned long long ld_key(const unsigned long long* p, int64_t i) {
    return __ldcs(p + i) & 0x7fffffffffffffffULL;
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
// lane has the same digit one lane adds them all; otherwise lanes with equal
// digits add once each. Called by the whole warp.
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

// Pass 1 over every value: the first-digit histogram (one per layer, shared
// by its problems; zeros counted in registers, other keys added to the
// shared-memory histogram one lane at a time), the smallest and largest key.
// The last block of a layer picks its problems' first digits and the list
// length; the last layer picked lays out the lists, greedily in layer order
// while they fit the budget.
__global__ void __launch_bounds__(kThreads, 5) first_pass_kernel(const double* __restrict__ ylt, int64_t n, int n_p,
                                                              const KParams kq, SelState* __restrict__ st,
                                                              LayerState* __restrict__ ls,
                                                              unsigned int* __restrict__ hist1,
                                                              unsigned long long* __restrict__ part_max,
                                                              unsigned int* __restrict__ tickets,
                                                              unsigned long long cand_budget) {
    extern __shared__ unsigned int sh_hist[];  // [kBins1]
    __shared__ unsigned long long sh_red_u[32];
    __shared__ bool sh_last;
    __shared__ unsigned long long sh_need[kThreads];
    const int j = blockIdx.y;
    const int n_layers = gridDim.y;
    for (int i = threadIdx.x; i < kBins1; i += blockDim.x) sh_hist[i] = 0;
    __syncthreads();
    const unsigned long long* row = reinterpret_cast<const unsigned long long*>(ylt) + (size_t)j * (size_t)n;
    // the thread's largest key and how often it holds it; the smallest key
    unsigned long long kmax = 0, cmax = 0, kinv = 0, zeros = 0;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kUnroll; i0 < n;
         i0 += (int64_t)gridDim.x * blockDim.x * kUnroll) {
        unsigned long long kv[kUnroll];
        bool valid[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x + threadIdx.x;
            valid[u] = i < n;
            kv[u] = valid[u] ? ld_key(row, i) : 0ULL;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const unsigned long long key = kv[u];
            if (valid[u]) {
                // zeros and the thread's running largest key (trials at the
                // aggregate cap) are counted in registers; a new largest key
                // hands the old one's count to the histogram
                if (key == 0ULL) {
                    ++zeros;
                } else if (key == kmax) {
                    ++cmax;
                } else if (key > kmax) {
                    if (cmax) atomicAdd(&sh_hist[kmax >> kShift1], (unsigned)cmax);
                    kmax = key;
                    cmax = 1;
                } else {
                    atomicAdd(&sh_hist[key >> kShift1], 1u);
                }
                kinv = max(kinv, ~key);
            }
        }
    }
    if (cmax) atomicAdd(&sh_hist[kmax >> kShift1], (unsigned)cmax);
    const unsigned long long a = block_max_u64(kmax, sh_red_u);
    __shared__ unsigned long long sh_bmax;
    if (threadIdx.x == 0) sh_bmax = a;
    __syncthreads();
    // how often the block holds its largest key
    const unsigned long long ca = block_sum_u64(kmax == sh_bmax ? cmax : 0ULL, sh_red_u);
    const unsigned long long b = block_max_u64(kinv, sh_red_u);
    const unsigned long long z = block_sum_u64(zeros, sh_red_u);
    if (threadIdx.x == 0) {
        part_max[2 * ((size_t)j * gridDim.x + blockIdx.x)] = a;
        part_max[2 * ((size_t)j * gridDim.x + blockIdx.x) + 1] = ca;
        atomicMax(&ls[j].kmax, a);
        atomicMax(&ls[j].kinv, b);
        if (z) {
            atomicAdd(&ls[j].cnt_zero, z);
            sh_hist[0] += (unsigned)z;
        }
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
    int lowest = kBins1;
    for (int q = 0; q < n_p; ++q) {
        SelState* sq = &st[j * n_p + q];
        if (hi == lo) {
            // a constant layer: every problem is decided by its one key
            if (threadIdx.x == 0) *sq = SelState{hi, kAllKeyBits, 1, kq.k[q]};
        } else {
            int bin;
            unsigned long long above;
            pick_digit(sh_hist, kBins1, kq.k[q], &bin, &above);
            lowest = min(lowest, bin);
            if (threadIdx.x == 0)
                *sq = SelState{(unsigned long long)bin << kShift1, (unsigned long long)(kBins1 - 1) << kShift1,
                               kq.k[q] - (long long)above, kq.k[q]};
        }
    }
    // how often the layer holds its largest key: the blocks holding it
    unsigned long long cm = 0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        if (__ldcg(&part_max[2 * ((size_t)j * gridDim.x + b)]) == hi)
            cm += __ldcg(&part_max[2 * ((size_t)j * gridDim.x + b) + 1]);
    cm = block_sum_u64(cm, sh_red_u);
    // list slots: every key at or above the lowest selected bucket other
    // than 0 and the largest key (counted, not listed)
    unsigned long long need = 0;
    if (hi != lo)
        for (int i = lowest + (int)threadIdx.x; i < kBins1; i += blockDim.x) need += sh_hist[i];
    need = block_sum_u64(need, sh_red_u);
    if (threadIdx.x == 0) {
        const unsigned long long cz = __ldcg(&ls[j].cnt_zero);
        unsigned long long need_sel = 0;  // or the keys of the selected buckets only
        if (hi != lo) {
            need -= cm + (lowest == 0 ? cz : 0ULL);
            bool max_sel = false, zero_sel = false;
            for (int q = 0; q < n_p; ++q) {
                const unsigned long long bq = st[j * n_p + q].prefix >> kShift1;
                bool seen = false;
                for (int r = 0; r < q; ++r) seen = seen || (st[j * n_p + r].prefix >> kShift1) == bq;
                if (!seen) need_sel += sh_hist[bq];
                max_sel = max_sel || bq == (hi >> kShift1);
                zero_sel = zero_sel || bq == 0;
            }
            need_sel -= (max_sel ? cm : 0ULL) + (zero_sel ? cz : 0ULL);
        }
        ls[j].cnt_max = cm;
        ls[j].need_sel = need_sel;
        ls[j].need = need;
        ls[j].lo_bucket = hi != lo ? (unsigned long long)lowest : 0ULL;
        ls[j].stage = hi != lo ? 1 : kPasses;
        tickets[j] = 0;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh_last = atomicAdd(&tickets[n_layers], 1u) == (unsigned)n_layers - 1;
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    // the last layer picked: the lists in layer order while they fit
    unsigned long long run = 0;
    for (int c0 = 0; c0 < n_layers; c0 += kThreads) {
        const int jj = c0 + threadIdx.x;
        sh_need[threadIdx.x] = jj < n_layers ? __ldcg(&ls[jj].need) : 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int t = 0; t < kThreads && c0 + t < n_layers; ++t) {
                LayerState& l = ls[c0 + t];
                const unsigned long long nd = sh_need[t], ns = __ldcg(&l.need_sel);
                const int mode = run + nd <= cand_budget ? kListAll : run + ns <= cand_budget ? kListSelected
                                                                                                : kListNone;
                const unsigned long long len = mode == kListAll ? nd : mode == kListSelected ? ns : 0ULL;
                l.compact = mode;
                l.need = len;
                l.cand_off = run;
                run += len;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) tickets[n_layers] = 0;
}

// Passes 2-7, one digit per layer and launch. Pass 2 (second) reads every
// value: it adds each layer's sum, counts the layer's largest keys and, for a
// layer with a list, writes the list; a layer without one histograms its
// next digit there. Later passes histogram each layer's next digit from its
// list or its row. Problems with the same prefix share the histogram of the
// first of them. The last block of a layer picks the digits; the keys
// counted instead of listed enter its histograms and extremes where they
// match.
template <int NQ>
__global__ void __launch_bounds__(kThreads, NQ == 2 ? 3 : 4) pass_kernel(const double* __restrict__ ylt, int64_t n, int n_p,
                                                        SelState* __restrict__ st, LayerState* __restrict__ ls,
                                                        unsigned long long* __restrict__ cand, bool second,
                                                        unsigned int* __restrict__ ghist,
                                                        unsigned long long* __restrict__ minmax,
                                                        unsigned long long* __restrict__ msum,
                                                        unsigned int* __restrict__ tickets) {
    extern __shared__ unsigned int sh_hist[];  // [n_p][1 << bits]
    __shared__ unsigned long long sh_red_u[32];
    __shared__ bool sh_last;
    __shared__ int sh_src[kMaxProbs];
    const int j = blockIdx.y;
    const unsigned lane = threadIdx.x & 31;
    const int stage = ls[j].stage;
    const int mode = ls[j].compact;
    const bool compact = mode != kListNone;
    const unsigned long long kmax_l = ls[j].kmax;
    // pass 2 always runs (the layer sums); later passes only while a digit is left
    if (stage >= kPasses && !second) return;  // the same for every block of the layer: no ticket
    const bool histo = stage < kPasses && !(second && compact);
    const int shift = pass_shift(min(stage, kPasses - 1)), bits = pass_bits(min(stage, kPasses - 1));
    const int nb = 1 << bits;
    unsigned long long pre[NQ], msk[NQ];
    bool done[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        pre[q] = q < n_p ? st[j * n_p + q].prefix : 1ULL;  // unused slots never match
        msk[q] = q < n_p ? st[j * n_p + q].mask : 0ULL;
        done[q] = !histo || q >= n_p || msk[q] == kAllKeyBits;
    }
    const bool from_row = second || !compact;
    const unsigned long long* src_vals = from_row
                                             ? reinterpret_cast<const unsigned long long*>(ylt) + (size_t)j * (size_t)n
                                             : cand + ls[j].cand_off;
    const int64_t len = from_row ? n : (int64_t)min((unsigned long long)ls[j].cand_n, ls[j].need);
    const bool writing = second && compact && stage < kPasses;  // pass 2 writes the layer's list
    unsigned long long* my_cand = cand + ls[j].cand_off;
    const unsigned long long cap = ls[j].need;
    const unsigned long long lo_bucket = ls[j].lo_bucket;
    const int e_ref = ref_exp(kmax_l);
    int src[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        src[q] = q;
#pragma unroll
        for (int r = NQ - 1; r >= 0; --r)
            if (r < q && !done[r] && !done[q] && pre[r] == pre[q] && msk[r] == msk[q]) src[q] = r;
        if (threadIdx.x == 0 && q < n_p) sh_src[q] = src[q];
    }
    // a block with no value to read (a short list) only takes its ticket
    const bool idle = (int64_t)blockIdx.x * blockDim.x * kUnroll >= len;
    if (histo && !idle)
        for (int i = threadIdx.x; i < n_p * nb; i += blockDim.x) sh_hist[i] = 0;
    unsigned long long kmx[NQ], kiv[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        kmx[q] = 0;
        kiv[q] = 0;
    }
    Fix sum{0, 0};
    __syncthreads();
    const unsigned dmask = (unsigned)nb - 1u;
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kUnroll; i0 < len;
         i0 += (int64_t)gridDim.x * blockDim.x * kUnroll) {
        unsigned long long kv[kUnroll];  // keys (0 past the end)
        bool valid[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x + threadIdx.x;
            valid[u] = i < len;
            kv[u] = valid[u] ? ld_key(src_vals, i) : 0ULL;
        }
        if (writing) {
            // the step's list entries: one counter update per warp and step
            unsigned m[kUnroll];
            unsigned tot = 0;
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const unsigned long long key = kv[u];
                bool in = key >> kShift1 >= lo_bucket;
                if (mode == kListSelected) {
                    in = false;
#pragma unroll
                    for (int q = 0; q < NQ; ++q)
                        in = in || (q < n_p && msk[q] != kAllKeyBits && (key & msk[q]) == pre[q]);
                }
                m[u] = __ballot_sync(0xffffffffu, in && key != 0ULL && key != kmax_l);
                tot += __popc(m[u]);
            }
            if (tot) {
                unsigned int base = 0;
                if (lane == 0) base = atomicAdd(&ls[j].cand_n, tot);
                base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    const unsigned long long slot = (unsigned long long)base + __popc(m[u] & lt_mask);
                    if (((m[u] >> lane) & 1u) && slot < cap) my_cand[slot] = kv[u];
                    base += __popc(m[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const unsigned long long key = kv[u];
            if (second) fix_add(sum, key, e_ref);  // invalid slots add 0
            if (histo) {
                const unsigned dig = (unsigned)(key >> shift) & dmask;
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    if (q < n_p && !done[q] && src[q] == q) {  // the same for the whole block
                        const bool hit = valid[u] && (key & msk[q]) == pre[q];
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
            }
        }
    }
    if (second) fix_block_atomic(msum + 2 * (size_t)j, sum);
    if (!histo) return;  // nothing to pick: no ticket is taken by any block of the layer
    unsigned int* gh = ghist + ((size_t)j * n_p) * kMaxBins;
    if (!idle) {
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
        for (int i = threadIdx.x; i < n_p * nb; i += blockDim.x) {
            const int q = i >> bits, b = i & (int)dmask;
            const unsigned c = sh_hist[sh_src[q] * nb + b];  // zero for a decided problem
            if (c) atomicAdd(&gh[(size_t)q * kMaxBins + b], c);
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh_last = atomicAdd(&tickets[j], 1u) == gridDim.x - 1;
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    // keys counted instead of listed take part where they match
    const bool virt = !from_row;
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
    if (threadIdx.x == 0) {
        ls[j].stage = stage + 1;
        tickets[j] = 0;
    }
}

// The tail, fused with the final reduction. Per problem, the keys above its
// k-th largest key and their exact fixed-point sum, from the layer's list
// (plus the counted largest keys when they lie above it) or from its row;
// nothing is read for a problem whose k-th largest is the layer's largest
// key. Blocks add their integer sums with atomics. The last block of the grid
// converts every problem's sums (one warp per problem) and writes mean, PML
// and TVaR (and, if asked, each layer's sum).
template <int NQ>
__global__ void __launch_bounds__(kThreads, NQ <= 4 ? 4 : 2) tail_kernel(const double* __restrict__ ylt, int64_t n, int n_p,
                                                        const SelState* __restrict__ st,
                                                        const LayerState* __restrict__ ls,
                                                        const unsigned long long* __restrict__ cand,
                                                        const unsigned long long* __restrict__ msum,
                                                        unsigned long long* __restrict__ tsum,
                                                        unsigned int* __restrict__ ticket, double* mean, double* pml,
                                                        double* tvar, double* sum_out) {
    __shared__ unsigned long long sh_red_u[32];
    __shared__ bool sh_last;
    const int j = blockIdx.y;
    const int n_layers = gridDim.y;
    const bool compact = ls[j].compact == kListAll;  // the list holds every key above the k-th largest
    const unsigned long long kmax_l = ls[j].kmax;
    const int e_ref = ref_exp(kmax_l);
    unsigned long long thr[NQ];
    bool live[NQ];
    bool any_live = false;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        thr[q] = q < n_p ? st[j * n_p + q].prefix : ~0ULL;
        live[q] = q < n_p && thr[q] < kmax_l;  // nothing lies above the layer's largest key
        any_live = any_live || live[q];
    }
    const unsigned long long* src_vals = compact
                                             ? cand + ls[j].cand_off
                                             : reinterpret_cast<const unsigned long long*>(ylt) + (size_t)j * (size_t)n;
    const int64_t len = !any_live ? 0
                        : compact ? (int64_t)min((unsigned long long)ls[j].cand_n, ls[j].need) : n;
    Fix s[NQ];
    unsigned long long c[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        s[q] = Fix{0, 0};
        c[q] = 0;
    }
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x * kUnroll; i0 < len;
         i0 += (int64_t)gridDim.x * blockDim.x * kUnroll) {
        unsigned long long kv[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int64_t i = i0 + (int64_t)u * blockDim.x + threadIdx.x;
            kv[u] = i < len ? ld_key(src_vals, i) : 0ULL;  // 0: never above a k-th largest key
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const unsigned long long key = kv[u];
            unsigned long long a0, a1;
            fix_words(key, e_ref, a0, a1);
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (live[q] && key > thr[q]) {
                    fix_add2(s[q], a0, a1);
                    c[q] += 1;
                }
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        if (!live[q]) continue;
        unsigned long long* g = tsum + 3 * ((size_t)j * n_p + q);
        fix_block_atomic(g, s[q]);
        const unsigned long long cc = block_sum_u64(c[q], sh_red_u);
        if (threadIdx.x == 0 && cc) atomicAdd(g + 2, cc);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) sh_last = atomicAdd(ticket, 1u) == gridDim.x * gridDim.y - 1;
    __syncthreads();
    if (!sh_last) return;
    __threadfence();
    // every problem's sums converted, one thread per problem
    for (int i = threadIdx.x; i < n_layers * n_p; i += blockDim.x) {
        const int jj = i / n_p, q = i % n_p;
        const SelState sq = st[i];
        const unsigned long long kmx = __ldcg(&ls[jj].kmax);
        const int er = ref_exp(kmx);
        if (q == 0) {
            const Fix ms{__ldcg(msum + 2 * (size_t)jj), __ldcg(msum + 2 * (size_t)jj + 1)};
            const double total = fix_value(ms, er);
            if (mean) mean[jj] = total / (double)n;
            if (sum_out) sum_out[jj] = total;
        }
        const unsigned long long* g = tsum + 3 * (size_t)i;
        Fix f{__ldcg(g), __ldcg(g + 1)};
        unsigned long long cnt = __ldcg(g + 2);
        if (__ldcg(&ls[jj].compact) == kListAll && kmx > sq.prefix) {
            // the layer's largest keys were counted, not listed
            const unsigned long long cm = __ldcg(&ls[jj].cnt_max);
            fix_add_times(f, kmx, er, cm);
            cnt += cm;
        }
        const double v = __longlong_as_double((long long)sq.prefix);
        if (pml) pml[i] = v;
        if (tvar) tvar[i] = (fix_value(f, er) + (double)(sq.k - (long long)cnt) * v) / (double)sq.k;
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
    size_t pmax, st, ls, hist1, hist, minmax, tickets, msum, tsum, cand;
    size_t zero, zero_bytes, total;
};

MetricsLayout metrics_layout(int32_t n_layers, int32_t n_p, int nblk, uint64_t cand_slots) {
    const size_t L = (size_t)n_layers, np = (size_t)n_layers * n_p;
    MetricsLayout m{};
    m.pmax = 0;
    m.st = align256(m.pmax + sizeof(unsigned long long) * 2 * L * (size_t)nblk);
    m.ls = align256(m.st + sizeof(SelState) * np);
    m.hist1 = align256(m.ls + sizeof(LayerState) * L);
    m.hist = align256(m.hist1 + sizeof(unsigned int) * kBins1 * L);
    m.minmax = align256(m.hist + sizeof(unsigned int) * kMaxBins * np);
    m.tickets = align256(m.minmax + sizeof(unsigned long long) * 2 * np);
    m.msum = align256(m.tickets + sizeof(unsigned int) * (L + 2));
    m.tsum = align256(m.msum + sizeof(unsigned long long) * 2 * L);
    m.cand = align256(m.tsum + sizeof(unsigned long long) * 3 * np);
    m.zero = m.ls;
    m.zero_bytes = m.cand - m.ls;
    m.total = align256(m.cand + sizeof(unsigned long long) * (size_t)cand_slots);
    return m;
}

// Candidate slots the allocating path reserves: an eighth of the YLT (the
// lists hold the top few percent of a layer's trials, its largest key left
// out), at least 65,536, at most the whole YLT.
uint64_t default_cand_slots(int64_t n, int32_t n_layers) {
    const uint64_t all = (uint64_t)n * (uint64_t)n_layers;
    return std::min<uint64_t>(all, std::max<uint64_t>(all / 8, 65536));
}

// The metric kernels over a caller's scratch laid out by metrics_layout:
// clear, pass 1, passes 2-7, the tail with the final reduction (nine steps
// on the stream, eight of them launches).
cudaError_t launch_metric_kernels(const double* ylt, int64_t n, int32_t n_layers, int32_t n_p, const KParams& kq,
                                  int nblk, char* w, const MetricsLayout& m, uint64_t cand_slots, double* mean,
                                  double* pml, double* tvar, double* sum_out, cudaStream_t s) {
    auto* pmax = (unsigned long long*)(w + m.pmax);
    auto* st = (SelState*)(w + m.st);
    auto* ls = (LayerState*)(w + m.ls);
    auto* hist1 = (unsigned int*)(w + m.hist1);
    auto* hist = (unsigned int*)(w + m.hist);
    auto* minmax = (unsigned long long*)(w + m.minmax);
    auto* tickets = (unsigned int*)(w + m.tickets);
    auto* msum = (unsigned long long*)(w + m.msum);
    auto* tsum = (unsigned long long*)(w + m.tsum);
    auto* cand = (unsigned long long*)(w + m.cand);
    cudaError_t err = cudaMemsetAsync(w + m.zero, 0, m.zero_bytes, s);
    if (err) return err;
    const dim3 grid(nblk, n_layers);
    first_pass_kernel<<<grid, kThreads, sizeof(unsigned int) * kBins1, s>>>(ylt, n, n_p, kq, st, ls, hist1, pmax,
                                                                            tickets, cand_slots);
    if ((err = cudaGetLastError())) return err;
    // the probability loops are compiled for 1, 2, 4 or 8 problems per layer
    auto pass_k = n_p <= 1 ? pass_kernel<1> : n_p <= 2 ? pass_kernel<2> : n_p <= 4 ? pass_kernel<4> : pass_kernel<8>;
    auto tail_k = n_p <= 1 ? tail_kernel<1> : n_p <= 2 ? tail_kernel<2> : n_p <= 4 ? tail_kernel<4> : tail_kernel<8>;
    const size_t shm = sizeof(unsigned int) * (size_t)n_p * kMaxBins;
    if (shm > 48 * 1024 && (err = cudaFuncSetAttribute(pass_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm)))
        return err;
    // pass 2, then one launch per digit a layer's list may still need
    for (int i = 0; i < kPasses; ++i) {
        pass_k<<<grid, kThreads, shm, s>>>(ylt, n, n_p, st, ls, cand, i == 0, hist, minmax, msum, tickets);
        if ((err = cudaGetLastError())) return err;
    }
    tail_k<<<grid, kThreads, 0, s>>>(ylt, n, n_p, st, ls, cand, msum, tsum, tickets + n_layers + 1, mean, pml, tvar,
                                     sum_out);
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

size_t metrics_scratch_bytes(int64_t n, int32_t n_layers, int32_t n_p) {
    return metrics_layout(n_layers, n_p, blocks_per_layer(n, n_layers), default_cand_slots(n, n_layers)).total;
}

cudaError_t metrics_run_k(const double* ylt, int64_t n, int32_t n_layers, const int64_t* k, int32_t n_p,
                          double* mean, double* pml, double* tvar, double* sum_out, cudaStream_t s,
                          void* scratch, size_t scratch_bytes) {
    const int nblk = blocks_per_layer(n, n_layers);
    const uint64_t slots = default_cand_slots(n, n_layers);
    const MetricsLayout m = metrics_layout(n_layers, n_p, nblk, slots);
    char* w = static_cast<char*>(scratch);
    const bool own = !w || scratch_bytes < m.total;
    cudaError_t err = own ? cudaMallocAsync((void**)&w, m.total, s) : cudaSuccess;
    if (err != cudaSuccess) return err;
    KParams kq = {};
    for (int q = 0; q < n_p; ++q) kq.k[q] = std::min<int64_t>(n, std::max<int64_t>(1, k[q]));
    err = launch_metric_kernels(ylt, n, n_layers, n_p, kq, nblk, w, m, slots, mean, pml, tvar, sum_out, s);
    const cudaError_t e2 = own ? cudaFreeAsync(w, s) : cudaSuccess;
    return err ? err : e2;
}

cudaError_t metrics_run(const double* ylt, int64_t n, int32_t n_layers, const double* probs, int32_t n_p,
                        double* mean, double* pml, double* tvar, cudaStream_t s, void* scratch,
                        size_t scratch_bytes) {
    int64_t k[kMaxProbs];
    for (int q = 0; q < n_p; ++q) k[q] = tail_count(probs[q], n);
    return metrics_run_k(ylt, n, n_layers, k, n_p, mean, pml, tvar, nullptr, s, scratch, scratch_bytes);
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
    const MetricsLayout fixed = metrics_layout(n_layers, n_p, nblk, 0);
    if (fixed.total > (size_t)ART_METRICS_NOALLOC_SCRATCH_BYTES) return ART_EINVAL;
    const uint64_t slots = std::min<uint64_t>(((size_t)ART_METRICS_NOALLOC_SCRATCH_BYTES - fixed.total) / 8,
                                              default_cand_slots(n_trials, n_layers));
    const MetricsLayout m = metrics_layout(n_layers, n_p, nblk, slots);
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

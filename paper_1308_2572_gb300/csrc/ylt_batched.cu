// ylt_batched.cu -- one persistent launch for every layer of a portfolio
// (Section II, Algorithm 1 over all layers at once; Section III's direct-
// access tables, one pool-wide event-major table shared by all layers).
//
// Layout: the pool table is [C][NPOOL] (NPOOL = 32 * EPL >= n_elt, EPL a
// power of two): row i holds event i's loss in every ELT of the pool, so a
// warp reads one event's whole row with one coalesced load of NPOOL values,
// lane l holding ELTs l*EPL .. l*EPL+EPL-1.
//
// Per event: the warp ballots which of its values are non-zero (an absent
// loss is 0 and F_e(0) = 0 since D_e >= 0, so zeros contribute nothing and
// are skipped exactly); for each non-zero (ELT e, loss y), broadcast by a
// shuffle, every lane applies F_e(y) once and adds it to the per-event sums
// of the layers it owns that cover e (a per-(ELT, lane) bit mask in shared
// memory). Layers are spread over (lane, slot) pairs, SLOTS per lane, so each
// lane ends a trial holding the FP64 aggregates of its own layers and no
// cross-lane reduction is needed. A tile of 32 * SLOTS layers runs per work
// unit; portfolios with more layers run several layer tiles.
//
// Scheduling: a persistent grid (SM count x resident CTAs) whose warps pull
// work units (layer tile x trial tile) from an atomic counter; trials of
// uneven length balance dynamically. No warp ever waits on another.
//
// Precision: V = float is the mixed form (FP32 losses and per-event sums; the
// per-slot aggregate is a compensated FP32 pair, Knuth's two-sum, folded into
// FP64 at the end of the trial, where the aggregate terms apply in FP64);
// V = double is the all-FP64 form over an FP64 pool table, with the aggregate
// summed in FP64 event by event.
#include "art_internal.cuh"

namespace art {

template <typename V, int EPL>
__device__ __forceinline__ void load_row(const V* __restrict__ p, V (&v)[EPL]) {
    if constexpr (sizeof(V) == 4 && EPL >= 4) {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int i = 0; i < EPL / 4; ++i) {
            const float4 w = __ldg(q + i);
            v[4 * i + 0] = w.x;
            v[4 * i + 1] = w.y;
            v[4 * i + 2] = w.z;
            v[4 * i + 3] = w.w;
        }
    } else if constexpr (sizeof(V) == 4 && EPL == 2) {
        const float2 w = __ldg(reinterpret_cast<const float2*>(p));
        v[0] = w.x;
        v[1] = w.y;
    } else if constexpr (sizeof(V) == 8 && EPL >= 2) {
        const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
        for (int i = 0; i < EPL / 2; ++i) {
            const double2 w = __ldg(q + i);
            v[2 * i + 0] = w.x;
            v[2 * i + 1] = w.y;
        }
    } else {
        v[0] = __ldg(p);
    }
}

__device__ __forceinline__ float fin_v(float y, float m, float d, float l) { return fin_f32(y, m, d, l); }
__device__ __forceinline__ double fin_v(double y, double m, double d, double l) { return fin_f64(y, m, d, l); }
__device__ __forceinline__ float xl_v(float v, float r, float l) { return xl_f32(v, r, l); }
__device__ __forceinline__ double xl_v(double v, double r, double l) { return xl_f64(v, r, l); }

// Per-slot aggregate: FP32 values go into a compensated FP32 pair (two-sum),
// FP64 values straight into an FP64 sum.
struct AggF32 {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float v) {
        const float t = hi + v;
        const float bp = t - hi;
        lo += (hi - (t - bp)) + (v - bp);
        hi = t;
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
struct AggF64 {
    double s = 0.0;
    __device__ __forceinline__ void add(double v) { s += v; }
    __device__ __forceinline__ double value() const { return s; }
};
template <typename V> struct AggOf;
template <> struct AggOf<float> { using type = AggF32; };
template <> struct AggOf<double> { using type = AggF64; };

template <typename V, int EPL, int SLOTS, int U>
__global__ void __launch_bounds__(256) ylt_batched_kernel(const BatchedArgs a, const YetArgs y,
                                                          const int32_t trial_tile, const int64_t n_ttiles,
                                                          unsigned int* __restrict__ counter,
                                                          double* __restrict__ ylt,
                                                          uint8_t* __restrict__ branch,
                                                          int* __restrict__ flags) {
    constexpr int NPOOL = 32 * EPL;
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    V* s_m = reinterpret_cast<V*>(smem);
    V* s_d = s_m + NPOOL;
    V* s_l = s_d + NPOOL;
    uint8_t* s_memb = reinterpret_cast<uint8_t*>(s_l + NPOOL);  // [n_tiles][NPOOL][32]

    for (int i = threadIdx.x; i < NPOOL; i += blockDim.x) {
        if constexpr (sizeof(V) == 4) {
            s_m[i] = a.elt_terms[i];
            s_d[i] = a.elt_terms[NPOOL + i];
            s_l[i] = a.elt_terms[2 * NPOOL + i];
        } else {
            s_m[i] = a.elt_terms64[i];
            s_d[i] = a.elt_terms64[NPOOL + i];
            s_l[i] = a.elt_terms64[2 * NPOOL + i];
        }
    }
    {
        const int n16 = a.n_tiles * NPOOL * 32 / 16;
        const uint4* src = reinterpret_cast<const uint4*>(a.memb);
        uint4* dst = reinterpret_cast<uint4*>(s_memb);
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const V* __restrict__ pool = reinterpret_cast<const V*>(a.pool);
    const int64_t n_units = (int64_t)a.n_tiles * n_ttiles;
    bool bad_id = false, bad_off_seen = false;

    for (;;) {
        unsigned int unit = 0;
        if (lane == 0) unit = atomicAdd(counter, 1u);
        unit = __shfl_sync(FULL, unit, 0);
        if ((int64_t)unit >= n_units) break;
        const int tile = (int)((int64_t)unit / n_ttiles);
        const int64_t t0 = ((int64_t)unit % n_ttiles) * trial_tile;
        const int64_t t1 = min(t0 + (int64_t)trial_tile, y.n_trials);

        int32_t jl[SLOTS];
        V occ_r[SLOTS], occ_l[SLOTS];
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
            jl[s] = a.slot_layer[(tile * SLOTS + s) * 32 + lane];
            occ_r[s] = jl[s] >= 0 ? (V)a.occ[2 * jl[s]] : V(0);
            occ_l[s] = jl[s] >= 0 ? (V)a.occ[2 * jl[s] + 1] : V(0);
        }
        const uint8_t* memb = s_memb + (size_t)tile * NPOOL * 32;

        for (int64_t t = t0; t < t1; ++t) {
            int64_t b, e;
            bool bad_off;
            trial_range(y, t, b, e, bad_off);
            bad_off_seen |= bad_off;
            typename AggOf<V>::type S[SLOTS];

            for (int64_t d0 = b; d0 < e; d0 += 32) {
                const int cnt = (int)min((int64_t)32, e - d0);
                const int32_t myid = lane < cnt ? ld_stream(y.ids + d0 + lane) : 0;
                for (int ev0 = 0; ev0 < cnt; ev0 += U) {
                    V v[U][EPL];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int ev = ev0 + u;
                        const int32_t id = __shfl_sync(FULL, myid, ev & 31);
                        const bool live = ev < cnt;
                        const bool ok = live && (unsigned)id < (unsigned)y.catalogue;
                        if (live && !ok) bad_id = true;
                        if (ok) {
                            load_row<V, EPL>(pool + (size_t)id * NPOOL + lane * EPL, v[u]);
                        } else {
#pragma unroll
                            for (int k = 0; k < EPL; ++k) v[u][k] = V(0);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        V x[SLOTS];
#pragma unroll
                        for (int s = 0; s < SLOTS; ++s) x[s] = V(0);
#pragma unroll
                        for (int k = 0; k < EPL; ++k) {
                            unsigned mk = __ballot_sync(FULL, v[u][k] != V(0));
                            while (mk) {
                                const int src = __ffs(mk) - 1;
                                mk &= mk - 1;
                                const V yv = __shfl_sync(FULL, v[u][k], src);
                                const int el = src * EPL + k;
                                const V f = fin_v(yv, s_m[el], s_d[el], s_l[el]);
                                const unsigned bits = memb[el * 32 + lane];
#pragma unroll
                                for (int s = 0; s < SLOTS; ++s)
                                    if (bits & (1u << s)) x[s] += f;
                            }
                        }
#pragma unroll
                        for (int s = 0; s < SLOTS; ++s) {
                            const V o = xl_v(x[s], occ_r[s], occ_l[s]);
                            if (o > V(0)) S[s].add(o);
                        }
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < SLOTS; ++s) {
                const int32_t j = jl[s];
                if (j >= 0) {
                    const double ar = a.agg[2 * j], al = a.agg[2 * j + 1];
                    const double sum = S[s].value();
                    const size_t w = (size_t)j * (size_t)y.n_trials + (size_t)t;
                    ylt[w] = xl_f64(sum, ar, al);
                    if (branch) branch[w] = agg_branch(sum, ar, al);
                }
            }
        }
    }
    if (bad_id) atomicOr(flags + kFlagIdRange, 1);
    if (bad_off_seen && lane == 0) atomicOr(flags + kFlagBadOffsets, 1);
}

template <typename V, int EPL, int SLOTS, int U>
static cudaError_t launch_cfg(art_portfolio* p, const BatchedArgs& a, const YetArgs& y, double* ylt,
                              uint8_t* branch, cudaStream_t s) {
    auto kern = ylt_batched_kernel<V, EPL, SLOTS, U>;
    const size_t smem = 3 * (size_t)(32 * EPL) * sizeof(V) + (size_t)a.n_tiles * (32 * EPL) * 32;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int threads = (p->cta_threads > 0 && p->cta_threads <= 256) ? p->cta_threads : 256;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int32_t tt = p->trial_tile > 0 ? p->trial_tile : 4;
    const int64_t n_ttiles = (y.n_trials + tt - 1) / tt;
    if ((int64_t)a.n_tiles * n_ttiles >= 0xffffffffLL) return cudaErrorInvalidValue;
    int64_t grid = (int64_t)p->num_sms * per_sm;
    const int64_t warps_needed = (int64_t)a.n_tiles * n_ttiles;
    const int64_t grid_needed = (warps_needed + threads / 32 - 1) / (threads / 32);
    if (grid > grid_needed) grid = grid_needed;
    if (grid < 1) grid = 1;
    err = cudaMemsetAsync(p->d_work_counter, 0, sizeof(unsigned int), s);
    if (err != cudaSuccess) return err;
    kern<<<(unsigned)grid, threads, smem, s>>>(a, y, tt, n_ttiles, p->d_work_counter, ylt, branch, p->d_flags);
    return cudaGetLastError();
}

template <typename V, int EPL>
static cudaError_t launch_slots(art_portfolio* p, const BatchedArgs& a, const YetArgs& y, double* ylt,
                                uint8_t* branch, cudaStream_t s) {
    constexpr int U = sizeof(V) == 4 ? (EPL <= 8 ? 4 : 2) : (EPL <= 4 ? 4 : 2);
    switch (a.slots) {
        case 2: return launch_cfg<V, EPL, 2, U>(p, a, y, ylt, branch, s);
        case 4: return launch_cfg<V, EPL, 4, U>(p, a, y, ylt, branch, s);
        case 8: return launch_cfg<V, EPL, 8, U>(p, a, y, ylt, branch, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename V>
static cudaError_t launch_epl(art_portfolio* p, const BatchedArgs& a, const YetArgs& y, double* ylt,
                              uint8_t* branch, cudaStream_t s) {
    switch (a.pool_np / 32) {
        case 1: return launch_slots<V, 1>(p, a, y, ylt, branch, s);
        case 2: return launch_slots<V, 2>(p, a, y, ylt, branch, s);
        case 4: return launch_slots<V, 4>(p, a, y, ylt, branch, s);
        case 8: return launch_slots<V, 8>(p, a, y, ylt, branch, s);
        case 16: return launch_slots<V, 16>(p, a, y, ylt, branch, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batched(art_portfolio* p, const YetArgs& y, double* ylt, uint8_t* branch, bool fp64,
                           cudaStream_t s) {
    if (y.n_trials == 0) return cudaSuccess;
    BatchedArgs a;
    a.pool = fp64 ? (const void*)p->pool64 : (const void*)p->pool;
    a.elt_terms = p->d_elt_terms;
    a.elt_terms64 = p->d_elt_terms64;
    a.memb = p->d_memb;
    a.slot_layer = p->d_slot_layer;
    a.occ = p->d_occ;
    a.agg = p->d_agg;
    a.pool_np = p->pool_np;
    a.n_layers = p->n_layers;
    a.n_tiles = p->n_tiles;
    a.slots = p->slots;
    return fp64 ? launch_epl<double>(p, a, y, ylt, branch, s) : launch_epl<float>(p, a, y, ylt, branch, s);
}

}  // namespace art

// ylt_sparse.cu -- one persistent launch for every layer of a portfolio over a
// compressed ELT representation (Section II, Algorithm 1; Section VI names
// compressed in-memory representations as the next step after Section III's
// direct-access tables).
//
// Layout: an event-major CSR of the pool's non-zero losses: for event i,
// entries [ptr[i], ptr[i+1]) hold (loss, ELT) pairs in ELT order. A direct-
// access table holds zeros for every (event, ELT) without a loss; those add
// exactly nothing (F_e(0) = 0 since D_e >= 0), so the CSR gives the same
// per-event sums while reading about 8 bytes per non-zero loss instead of a
// whole table row. For the 256- and 512-ELT pools (about 1.5% non-zero) it is
// 70-130 MB, mostly L2-resident, against 2-4 GB of direct-access rows.
//
// Two mappings over a persistent grid whose warps pull work units (layer
// tile x trial tile) from an atomic counter, a warp taking one trial at a
// time; the autotuner picks one (art_autotune), the default is "scatter" for
// tiles of 64 layers and "broadcast" for larger ones.
//
// Broadcast: lane l owns the layers of slots s at (lane l, slot s). Per group
// of 32 events each lane reads its event's CSR range; for each event with
// entries, in trial order, the warp reads the entries (one address for all
// lanes), every lane applies F_e and adds it to its slots whose layer covers
// the ELT (a per-(ELT, lane) bit mask), then applies the occurrence terms.
//
// Scatter: 32 events per group. Phase 1: lane l walks the CSR entries of event l (in ELT order),
// applies F_e to each loss and adds it to the event's per-layer sums in its
// own row of a [32 events][layers] FP32 block in shared memory, through the
// ELT's list of covering layers in the tile. Each row has one writer, so the
// sums need no atomics and are formed in ELT order (deterministic). Phase 2:
// lane l owns the layers of slots s at (lane l, slot s); for each event of
// the group that had entries, in trial order, it reads the event's sums for
// its layers, applies the occurrence terms, adds the result to its per-slot
// aggregate (a compensated FP32 pair, two-sum) and clears the entry. At the
// end of the trial the pairs are folded into FP64 and the aggregate terms are
// applied in FP64.
#include <algorithm>

#include "art_internal.cuh"

namespace art {

namespace {

constexpr int kSparseThreads = 256;


__device__ __forceinline__ void two_sum_acc(float& s, float& e, float v) {
    const float t = s + v;
    const float bp = t - s;
    const float err = (s - (t - bp)) + (v - bp);
    s = t;
    e += err;
}

template <int SLOTS>
__global__ void __launch_bounds__(kSparseThreads) ylt_sparse_scatter_kernel(const SparseArgs a, const YetArgs y,
                                                                   const int32_t trial_tile, const int64_t n_ttiles,
                                                                   unsigned int* __restrict__ counter,
                                                                   double* __restrict__ ylt,
                                                                   uint8_t* __restrict__ branch,
                                                                   int* __restrict__ flags) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int LT = 32 * SLOTS;  // layers per tile
    constexpr int XS = LT + 1;      // row stride of the accumulator block (bank spread)
    extern __shared__ __align__(16) unsigned char smem[];
    float4* s_terms = reinterpret_cast<float4*>(smem);                                  // [pool_np]
    uint16_t* s_off = reinterpret_cast<uint16_t*>(s_terms + a.pool_np);                 // [n_tiles][pool_np + 1]
    const size_t off_bytes = (((size_t)a.n_tiles * (a.pool_np + 1) * 2) + 15) & ~(size_t)15;
    uint8_t* s_lay = reinterpret_cast<uint8_t*>(s_off) + off_bytes;                     // [n_tiles][tl_stride]
    float* s_x = reinterpret_cast<float*>(s_lay + (size_t)a.n_tiles * a.tl_stride);    // [warps][32][XS]
    for (int i = threadIdx.x; i < a.pool_np; i += blockDim.x)
        s_terms[i] = make_float4(a.elt_terms[i], a.elt_terms[a.pool_np + i], a.elt_terms[2 * a.pool_np + i], 0.f);
    for (int i = threadIdx.x; i < a.n_tiles * (a.pool_np + 1); i += blockDim.x) s_off[i] = a.tl_off[i];
    {
        const uint4* src = reinterpret_cast<const uint4*>(a.tl_lay);
        uint4* dst = reinterpret_cast<uint4*>(s_lay);
        for (int i = threadIdx.x; i < a.n_tiles * a.tl_stride / 16; i += blockDim.x) dst[i] = src[i];
    }
    const int n_warps_cta = blockDim.x >> 5;
    for (int i = threadIdx.x; i < n_warps_cta * 32 * XS; i += blockDim.x) s_x[i] = 0.0f;
    __syncthreads();

    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float* xw = s_x + (size_t)wib * 32 * XS;  // this warp's block; row l belongs to lane l in phase 1
    const SparseEntry* __restrict__ entries = reinterpret_cast<const SparseEntry*>(a.entries);
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
        float occ_r[SLOTS], occ_l[SLOTS];
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
            jl[s] = a.slot_layer[(tile * SLOTS + s) * 32 + lane];
            occ_r[s] = jl[s] >= 0 ? a.occ[2 * jl[s]] : 0.0f;
            occ_l[s] = jl[s] >= 0 ? a.occ[2 * jl[s] + 1] : 0.0f;
        }
        const uint16_t* off = s_off + (size_t)tile * (a.pool_np + 1);
        const uint8_t* lay = s_lay + (size_t)tile * a.tl_stride;
        float* xr = xw + lane * XS;

        for (int64_t t = t0; t < t1; ++t) {
            int64_t b, e;
            bool bad_off;
            trial_range(y, t, b, e, bad_off);
            bad_off_seen |= bad_off;
            const int32_t* tid = y.ids + b;
            const int32_t n = (int32_t)(e - b);
            float hi[SLOTS], lo[SLOTS];
#pragma unroll
            for (int s = 0; s < SLOTS; ++s) {
                hi[s] = 0.0f;
                lo[s] = 0.0f;
            }
            int32_t nid = lane < n ? ld_stream(tid + lane) : -1;
            for (int32_t c0 = 0; c0 < n; c0 += 32) {
                const int32_t id = nid;
                // the next group's id is requested before this group's entries
                nid = c0 + 32 + lane < n ? ld_stream(tid + c0 + 32 + lane) : -1;
                const bool live = c0 + lane < n;
                const bool ok = live && (unsigned)id < (unsigned)y.catalogue;
                if (live && !ok) bad_id = true;
                uint32_t p0 = 0, p1 = 0;
                if (ok) {
                    p0 = __ldg(a.ptr + id);
                    p1 = __ldg(a.ptr + id + 1);
                }
                // phase 1: this lane's event into its own row
                for (uint32_t k = p0; k < p1; ++k) {
                    const SparseEntry en = entries[k];
                    const float4 tm = s_terms[en.elt];
                    const float f = fin_f32(en.loss, tm.x, tm.y, tm.z);
                    const int q1 = off[en.elt + 1];
                    for (int q = off[en.elt]; q < q1; ++q) xr[lay[q]] += f;
                }
                __syncwarp();
                // phase 2: each lane folds its layers' sums, event by event in trial order
                unsigned mask = __ballot_sync(FULL, p1 > p0);
                while (mask) {
                    const int ev = __ffs(mask) - 1;
                    mask &= mask - 1;
                    float* row = xw + ev * XS;
#pragma unroll
                    for (int s = 0; s < SLOTS; ++s) {
                        const float x = row[lane + 32 * s];
                        if (x != 0.0f) {
                            row[lane + 32 * s] = 0.0f;
                            const float o = xl_f32(x, occ_r[s], occ_l[s]);
                            if (o > 0.0f) two_sum_acc(hi[s], lo[s], o);
                        }
                    }
                }
                __syncwarp();
            }
#pragma unroll
            for (int s = 0; s < SLOTS; ++s) {
                const int32_t j = jl[s];
                if (j >= 0) {
                    const double S = (double)hi[s] + (double)lo[s];
                    const double ar = a.agg[2 * j], al = a.agg[2 * j + 1];
                    const size_t w = (size_t)j * (size_t)y.n_trials + (size_t)t;
                    ylt[w] = xl_f64(S, ar, al);
                    if (branch) branch[w] = agg_branch(S, ar, al);
                }
            }
        }
    }
    if (bad_id) atomicOr(flags + kFlagIdRange, 1);
    if (bad_off_seen && lane == 0) atomicOr(flags + kFlagBadOffsets, 1);
}

template <int SLOTS>
cudaError_t launch_scatter(art_portfolio* p, const SparseArgs& a, const YetArgs& y, double* ylt, uint8_t* branch,
                           cudaStream_t s) {
    auto kern = ylt_sparse_scatter_kernel<SLOTS>;
    const size_t base = (size_t)a.pool_np * 16 + ((((size_t)a.n_tiles * (a.pool_np + 1) * 2) + 15) & ~(size_t)15) +
                        (size_t)a.n_tiles * a.tl_stride;
    const size_t per_warp = (size_t)32 * (32 * SLOTS + 1) * 4;
    int warps = (p->cta_threads > 0 && p->cta_threads <= kSparseThreads) ? p->cta_threads / 32 : kSparseThreads / 32;
    while (warps > 1 && base + warps * per_warp > 100 * 1024) --warps;  // at least two CTAs per SM
    const size_t smem = base + warps * per_warp;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int threads = 32 * warps;
    int per_sm = 0;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem))) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int32_t tt = p->trial_tile > 0 ? p->trial_tile : 4;
    const int64_t n_ttiles = (y.n_trials + tt - 1) / tt;
    if ((int64_t)a.n_tiles * n_ttiles >= 0xffffffffLL) return cudaErrorInvalidValue;
    int64_t grid = (int64_t)p->num_sms * per_sm;
    const int64_t units = (int64_t)a.n_tiles * n_ttiles;
    grid = std::min<int64_t>(grid, (units + warps - 1) / warps);
    if (grid < 1) grid = 1;
    if ((err = cudaMemsetAsync(p->d_work_counter, 0, sizeof(unsigned int), s))) return err;
    kern<<<(unsigned)grid, threads, smem, s>>>(a, y, tt, n_ttiles, p->d_work_counter, ylt, branch, p->d_flags);
    return cudaGetLastError();
}

template <int SLOTS>
__global__ void __launch_bounds__(kSparseThreads) ylt_sparse_bcast_kernel(const SparseArgs a, const YetArgs y,
                                                                   const int32_t trial_tile, const int64_t n_ttiles,
                                                                   unsigned int* __restrict__ counter,
                                                                   double* __restrict__ ylt,
                                                                   uint8_t* __restrict__ branch,
                                                                   int* __restrict__ flags) {
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    float4* s_terms = reinterpret_cast<float4*>(smem);                       // [pool_np] m, D, Lim
    uint8_t* s_memb = reinterpret_cast<uint8_t*>(s_terms + a.pool_np);      // [n_tiles][pool_np][32]
    for (int i = threadIdx.x; i < a.pool_np; i += blockDim.x)
        s_terms[i] = make_float4(a.elt_terms[i], a.elt_terms[a.pool_np + i], a.elt_terms[2 * a.pool_np + i], 0.f);
    {
        const int n16 = a.n_tiles * a.pool_np * 32 / 16;
        const uint4* src = reinterpret_cast<const uint4*>(a.memb);
        uint4* dst = reinterpret_cast<uint4*>(s_memb);
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const SparseEntry* __restrict__ entries = reinterpret_cast<const SparseEntry*>(a.entries);
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
        float occ_r[SLOTS], occ_l[SLOTS];
#pragma unroll
        for (int s = 0; s < SLOTS; ++s) {
            jl[s] = a.slot_layer[(tile * SLOTS + s) * 32 + lane];
            occ_r[s] = jl[s] >= 0 ? a.occ[2 * jl[s]] : 0.0f;
            occ_l[s] = jl[s] >= 0 ? a.occ[2 * jl[s] + 1] : 0.0f;
        }
        const uint8_t* memb = s_memb + (size_t)tile * a.pool_np * 32;

        for (int64_t t = t0; t < t1; ++t) {
            int64_t b, e;
            bool bad_off;
            trial_range(y, t, b, e, bad_off);
            bad_off_seen |= bad_off;
            const int32_t* tid = y.ids + b;
            const int32_t n = (int32_t)(e - b);
            float hi[SLOTS], lo[SLOTS];
#pragma unroll
            for (int s = 0; s < SLOTS; ++s) {
                hi[s] = 0.0f;
                lo[s] = 0.0f;
            }
            int32_t nid = lane < n ? ld_stream(tid + lane) : -1;
            for (int32_t c0 = 0; c0 < n; c0 += 32) {
                const int32_t id = nid;
                // the next group's id is requested before this group's entries
                nid = c0 + 32 + lane < n ? ld_stream(tid + c0 + 32 + lane) : -1;
                const bool live = c0 + lane < n;
                const bool ok = live && (unsigned)id < (unsigned)y.catalogue;
                if (live && !ok) bad_id = true;
                uint32_t p0 = 0, p1 = 0;
                if (ok) {
                    p0 = __ldg(a.ptr + id);
                    p1 = __ldg(a.ptr + id + 1);
                }
                unsigned mask = __ballot_sync(FULL, p1 > p0);
                while (mask) {
                    const int ev = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const uint32_t q0 = __shfl_sync(FULL, p0, ev);
                    const uint32_t q1 = __shfl_sync(FULL, p1, ev);
                    float x[SLOTS];
#pragma unroll
                    for (int s = 0; s < SLOTS; ++s) x[s] = 0.0f;
                    for (uint32_t k = q0; k < q1; ++k) {
                        const SparseEntry en = entries[k];
                        const float4 tm = s_terms[en.elt];
                        const float f = fin_f32(en.loss, tm.x, tm.y, tm.z);
                        const unsigned bits = memb[en.elt * 32 + lane];
#pragma unroll
                        for (int s = 0; s < SLOTS; ++s)
                            if (bits & (1u << s)) x[s] += f;
                    }
#pragma unroll
                    for (int s = 0; s < SLOTS; ++s) {
                        const float o = xl_f32(x[s], occ_r[s], occ_l[s]);
                        if (o > 0.0f) two_sum_acc(hi[s], lo[s], o);
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < SLOTS; ++s) {
                const int32_t j = jl[s];
                if (j >= 0) {
                    const double S = (double)hi[s] + (double)lo[s];
                    const double ar = a.agg[2 * j], al = a.agg[2 * j + 1];
                    const size_t w = (size_t)j * (size_t)y.n_trials + (size_t)t;
                    ylt[w] = xl_f64(S, ar, al);
                    if (branch) branch[w] = agg_branch(S, ar, al);
                }
            }
        }
    }
    if (bad_id) atomicOr(flags + kFlagIdRange, 1);
    if (bad_off_seen && lane == 0) atomicOr(flags + kFlagBadOffsets, 1);
}

template <int SLOTS>
cudaError_t launch_bcast(art_portfolio* p, const SparseArgs& a, const YetArgs& y, double* ylt, uint8_t* branch,
                         cudaStream_t s) {
    auto kern = ylt_sparse_bcast_kernel<SLOTS>;
    const size_t smem = (size_t)a.pool_np * sizeof(float4) + (size_t)a.n_tiles * a.pool_np * 32;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const int threads = (p->cta_threads > 0 && p->cta_threads <= kSparseThreads) ? p->cta_threads : kSparseThreads;
    int per_sm = 0;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem))) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int32_t tt = p->trial_tile > 0 ? p->trial_tile : 4;
    const int64_t n_ttiles = (y.n_trials + tt - 1) / tt;
    if ((int64_t)a.n_tiles * n_ttiles >= 0xffffffffLL) return cudaErrorInvalidValue;
    int64_t grid = (int64_t)p->num_sms * per_sm;
    const int64_t units = (int64_t)a.n_tiles * n_ttiles;
    grid = std::min<int64_t>(grid, (units + threads / 32 - 1) / (threads / 32));
    if (grid < 1) grid = 1;
    if ((err = cudaMemsetAsync(p->d_work_counter, 0, sizeof(unsigned int), s))) return err;
    kern<<<(unsigned)grid, threads, smem, s>>>(a, y, tt, n_ttiles, p->d_work_counter, ylt, branch, p->d_flags);
    return cudaGetLastError();
}

template <int SLOTS>
cudaError_t launch_slots(art_portfolio* p, const SparseArgs& a, const YetArgs& y, double* ylt, uint8_t* branch,
                         cudaStream_t s) {
    const int mapping = p->sparse_mapping >= 0 ? p->sparse_mapping : (SLOTS == 2 ? 1 : 0);
    return mapping == 1 ? launch_scatter<SLOTS>(p, a, y, ylt, branch, s) : launch_bcast<SLOTS>(p, a, y, ylt, branch, s);
}

// CSR build, pass 1: per event, the number of ELTs with a non-zero loss.
__global__ void sparse_count_kernel(const float* __restrict__ src, int32_t catalogue, int32_t n_elt,
                                    uint32_t* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= catalogue) return;
    uint32_t c = 0;
    for (int e = 0; e < n_elt; ++e) c += src[(int64_t)e * catalogue + i] != 0.0f;
    cnt[i] = c;
}

// Exclusive scan of cnt[0..n) into ptr[0..n], one CTA (n up to a few million:
// each thread scans a contiguous run, then the runs' totals are scanned).
__global__ void sparse_scan_kernel(const uint32_t* __restrict__ cnt, int32_t n, uint32_t* __restrict__ ptr) {
    __shared__ uint32_t part[1024];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t per = ((int64_t)n + nt - 1) / nt;
    const int64_t b = tid * per, e = min((int64_t)n, b + per);
    uint32_t s = 0;
    for (int64_t i = b; i < e; ++i) s += cnt[i];
    part[tid] = s;
    __syncthreads();
    if (tid == 0) {
        uint32_t run = 0;
        for (int k = 0; k < nt; ++k) {
            const uint32_t v = part[k];
            part[k] = run;
            run += v;
        }
        ptr[n] = run;
    }
    __syncthreads();
    uint32_t run = part[tid];
    for (int64_t i = b; i < e; ++i) {
        ptr[i] = run;
        run += cnt[i];
    }
}

// CSR build, pass 2: the entries of event i in ELT order.
__global__ void sparse_fill_kernel(const float* __restrict__ src, int32_t catalogue, int32_t n_elt,
                                   const uint32_t* __restrict__ ptr, SparseEntry* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= catalogue) return;
    uint32_t k = ptr[i];
    for (int e = 0; e < n_elt; ++e) {
        const float v = src[(int64_t)e * catalogue + i];
        if (v != 0.0f) out[k++] = SparseEntry{v, e};
    }
}

}  // namespace

cudaError_t build_sparse(art_portfolio* p, const float* src, cudaStream_t s) {
    const int32_t C = p->catalogue;
    cudaError_t e;
    if ((e = cudaMalloc(&p->sp_ptr, sizeof(uint32_t) * ((size_t)C + 1)))) return e;
    uint32_t* cnt = nullptr;
    if ((e = cudaMalloc(&cnt, sizeof(uint32_t) * (size_t)C))) return e;
    const unsigned grid = (unsigned)((C + 255) / 256);
    sparse_count_kernel<<<grid, 256, 0, s>>>(src, C, p->n_elt, cnt);
    sparse_scan_kernel<<<1, 1024, 0, s>>>(cnt, C, p->sp_ptr);
    if ((e = cudaGetLastError())) {
        cudaFree(cnt);
        return e;
    }
    uint32_t total = 0;
    e = cudaMemcpyAsync(&total, p->sp_ptr + C, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (!e) e = cudaStreamSynchronize(s);
    cudaFree(cnt);
    if (e) return e;
    p->sp_nnz = total;
    if ((e = cudaMalloc(&p->sp_entries, sizeof(SparseEntry) * std::max<size_t>(1, total)))) return e;
    sparse_fill_kernel<<<grid, 256, 0, s>>>(src, C, p->n_elt, p->sp_ptr, reinterpret_cast<SparseEntry*>(p->sp_entries));
    p->sparse_bytes = (int64_t)(sizeof(uint32_t) * ((size_t)C + 1) + sizeof(SparseEntry) * (size_t)total);
    return cudaGetLastError();
}

cudaError_t launch_sparse(art_portfolio* p, const YetArgs& y, double* ylt, uint8_t* branch, cudaStream_t s) {
    if (y.n_trials == 0) return cudaSuccess;
    SparseArgs a;
    a.ptr = p->sp_ptr;
    a.entries = p->sp_entries;
    a.elt_terms = p->d_elt_terms;
    a.memb = p->d_memb;
    a.tl_off = p->d_tl_off;
    a.tl_lay = p->d_tl_lay;
    a.tl_stride = p->tl_stride;
    a.slot_layer = p->d_slot_layer;
    a.occ = p->d_occ;
    a.agg = p->d_agg;
    a.pool_np = p->pool_np;
    a.n_tiles = p->n_tiles;
    switch (p->slots) {
        case 2: return launch_slots<2>(p, a, y, ylt, branch, s);
        case 4: return launch_slots<4>(p, a, y, ylt, branch, s);
        case 8: return launch_slots<8>(p, a, y, ylt, branch, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace art

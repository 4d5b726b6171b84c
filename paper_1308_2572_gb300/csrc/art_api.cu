// art_api.cu -- the C ABI of include/art.h: validation, the preprocessing
// stage (building the direct-access tables in the kernels' layouts), dispatch
// to the kernels, host-buffer staging, CUDA-graph replay and status.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "art_internal.cuh"

namespace art {

static thread_local std::string g_last_cuda_error;

void set_last_error(cudaError_t e) {
    if (e != cudaSuccess) g_last_cuda_error = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e);
}

// Set (or clear, bytes == 0) a persisting access-policy window on a stream.
cudaError_t set_window(cudaStream_t s, const void* base, size_t bytes) {
    cudaStreamAttrValue v;
    std::memset(&v, 0, sizeof(v));
    if (bytes) {
        int dev = 0, max_win = 0, persist_max = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&max_win, cudaDevAttrMaxAccessPolicyWindowSize, dev);
        cudaDeviceGetAttribute(&persist_max, cudaDevAttrMaxPersistingL2CacheSize, dev);
        const size_t win = std::min(bytes, (size_t)max_win);
        v.accessPolicyWindow.base_ptr = const_cast<void*>(base);
        v.accessPolicyWindow.num_bytes = win;
        v.accessPolicyWindow.hitRatio = win ? (float)std::min(1.0, (double)persist_max / (double)win) : 0.0f;
        v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
        v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    }
    return cudaStreamSetAttribute(s, cudaStreamAttributeAccessPolicyWindow, &v);
}

}  // namespace art

using namespace art;

namespace {

__global__ void check_losses_kernel(const float* __restrict__ v, int64_t n, int* __restrict__ bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = v[i];
        if (!(x >= 0.0f) || !(x <= 3.4028234663852886e38f)) {  // negative, NaN or inf
            atomicOr(bad, 1);
            return;
        }
    }
}

art_status fail(cudaError_t e) {
    set_last_error(e);
    if (e == cudaErrorMemoryAllocation) return ART_ENOMEM;
    return ART_ECUDA;
}

bool finite_nonneg(double x) { return std::isfinite(x) && x >= 0.0; }
bool valid_limit(double x) { return !std::isnan(x) && x > 0.0; }  // +inf allowed

int pad_np(int n) {
    if (n <= 4) return 4;
    if (n <= 8) return 8;
    if (n <= 16) return 16;
    if (n <= 24) return 24;
    return 32;
}

// Round ELT and layer terms as the kernels apply them; false when invalid.
bool round_terms(int32_t n_elt, const float* m, const float* d, const float* l, int32_t n_layers,
                 const art_layer_terms* t, std::vector<float>& om, std::vector<float>& od, std::vector<float>& ol,
                 std::vector<float>& orr, std::vector<float>& orl, std::vector<double>& oar,
                 std::vector<double>& oal) {
    // NULL arrays keep the current values (partial updates)
    if (m) {
        om.assign(m, m + n_elt);
        for (float x : om)
            if (!finite_nonneg(x)) return false;
    }
    if (d) {
        od.assign(d, d + n_elt);
        for (float x : od)
            if (!finite_nonneg(x)) return false;
    }
    if (l) {
        ol.assign(l, l + n_elt);
        for (float x : ol)
            if (!valid_limit(x)) return false;
    }
    if (t) {
        orr.resize(n_layers);
        orl.resize(n_layers);
        oar.resize(n_layers);
        oal.resize(n_layers);
        for (int32_t j = 0; j < n_layers; ++j) {
            const art_layer_terms& x = t[j];
            if (!finite_nonneg(x.occ_ret) || !valid_limit(x.occ_lim) || !finite_nonneg(x.agg_ret) ||
                !valid_limit(x.agg_lim))
                return false;
            orr[j] = (float)x.occ_ret;
            orl[j] = (float)x.occ_lim;
            if (!std::isfinite(orr[j]) || !(orl[j] > 0.0f)) return false;  // overflow on rounding
            oar[j] = x.agg_ret;
            oal[j] = x.agg_lim;
        }
    }
    return true;
}

// Batched metadata: terms per pool column, (lane, slot) -> layer, and per
// (ELT, lane) the bit mask of the lane's slots whose layer covers the ELT.
cudaError_t upload_batched_terms(art_portfolio* p) {
    const int np = p->pool_np;
    std::vector<float> t32(3 * (size_t)np);
    std::vector<double> t64(3 * (size_t)np);
    for (int e = 0; e < np; ++e) {
        const bool real = e < p->n_elt;
        t32[e] = real ? p->mult[e] : 1.0f;
        t32[np + e] = real ? p->ded[e] : 0.0f;
        t32[2 * np + e] = real ? p->lim[e] : std::numeric_limits<float>::infinity();
        for (int k = 0; k < 3; ++k) t64[k * np + e] = (double)t32[k * np + e];
    }
    std::vector<float> occ(2 * (size_t)p->n_layers);
    std::vector<double> agg(2 * (size_t)p->n_layers);
    for (int j = 0; j < p->n_layers; ++j) {
        occ[2 * j] = p->occ_ret[j];
        occ[2 * j + 1] = p->occ_lim[j];
        agg[2 * j] = p->agg_ret[j];
        agg[2 * j + 1] = p->agg_lim[j];
    }
    cudaError_t e;
    if ((e = cudaMemcpy(p->d_elt_terms, t32.data(), sizeof(float) * t32.size(), cudaMemcpyHostToDevice))) return e;
    if ((e = cudaMemcpy(p->d_elt_terms64, t64.data(), sizeof(double) * t64.size(), cudaMemcpyHostToDevice))) return e;
    if ((e = cudaMemcpy(p->d_occ, occ.data(), sizeof(float) * occ.size(), cudaMemcpyHostToDevice))) return e;
    return cudaMemcpy(p->d_agg, agg.data(), sizeof(double) * agg.size(), cudaMemcpyHostToDevice);
}

}  // namespace

// Layer tile of the persistent kernels: layer j sits at (tile, slot, lane)
// with 32 * slots layers per tile; memb holds, per (tile, ELT, lane), the
// bits of the lane's slots whose layer covers the ELT.
cudaError_t art::set_layer_tile(art_portfolio* p, int32_t slots) {
    const int L = p->n_layers;
    const int per_tile = 32 * slots;
    const int n_tiles = (L + per_tile - 1) / per_tile;
    const int np = p->pool_np;
    std::vector<int32_t> slot_layer((size_t)n_tiles * slots * 32, -1);
    std::vector<uint8_t> memb((size_t)n_tiles * np * 32, 0);
    for (int j = 0; j < L; ++j) {
        const int tile = j / per_tile, r = j % per_tile, slot = r / 32, lane = r % 32;
        slot_layer[((size_t)tile * slots + slot) * 32 + lane] = j;
        for (int c = p->loff[j]; c < p->loff[j + 1]; ++c)
            memb[((size_t)tile * np + p->lids[c]) * 32 + lane] |= (uint8_t)(1u << slot);
    }
    // per tile, per ELT: the tile-local indices of the layers covering it, in
    // layer order (the sparse kernel's scatter lists)
    std::vector<std::vector<uint8_t>> lists((size_t)n_tiles * np);
    for (int j = 0; j < L; ++j)
        for (int c = p->loff[j]; c < p->loff[j + 1]; ++c)
            lists[(size_t)(j / per_tile) * np + p->lids[c]].push_back((uint8_t)(j % per_tile));
    size_t stride = 16;
    for (int t = 0; t < n_tiles; ++t) {
        size_t tot = 0;
        for (int e2 = 0; e2 < np; ++e2) tot += lists[(size_t)t * np + e2].size();
        stride = std::max(stride, (tot + 15) & ~(size_t)15);
    }
    std::vector<uint16_t> tl_off((size_t)n_tiles * (np + 1));
    std::vector<uint8_t> tl_lay((size_t)n_tiles * stride, 0);
    for (int t = 0; t < n_tiles; ++t) {
        uint16_t pos = 0;
        for (int e2 = 0; e2 < np; ++e2) {
            tl_off[(size_t)t * (np + 1) + e2] = pos;
            for (uint8_t v : lists[(size_t)t * np + e2]) tl_lay[(size_t)t * stride + pos++] = v;
        }
        tl_off[(size_t)t * (np + 1) + np] = pos;
    }
    int32_t* d_sl = nullptr;
    uint8_t* d_mb = nullptr;
    uint16_t* d_to = nullptr;
    uint8_t* d_tl = nullptr;
    cudaError_t e;
    auto cleanup = [&]() {
        cudaFree(d_sl);
        cudaFree(d_mb);
        cudaFree(d_to);
        cudaFree(d_tl);
    };
    if ((e = cudaMalloc(&d_sl, sizeof(int32_t) * slot_layer.size())) || (e = cudaMalloc(&d_mb, memb.size())) ||
        (e = cudaMalloc(&d_to, sizeof(uint16_t) * tl_off.size())) || (e = cudaMalloc(&d_tl, tl_lay.size()))) {
        cleanup();
        return e;
    }
    e = cudaMemcpy(d_sl, slot_layer.data(), sizeof(int32_t) * slot_layer.size(), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(d_mb, memb.data(), memb.size(), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(d_to, tl_off.data(), sizeof(uint16_t) * tl_off.size(), cudaMemcpyHostToDevice);
    if (!e) e = cudaMemcpy(d_tl, tl_lay.data(), tl_lay.size(), cudaMemcpyHostToDevice);
    if (e) {
        cleanup();
        return e;
    }
    cudaDeviceSynchronize();  // no launch may still read the old tile
    cudaFree(p->d_slot_layer);
    cudaFree(p->d_memb);
    cudaFree(p->d_tl_off);
    cudaFree(p->d_tl_lay);
    p->d_slot_layer = d_sl;
    p->d_memb = d_mb;
    p->d_tl_off = d_to;
    p->d_tl_lay = d_tl;
    p->tl_stride = (int32_t)stride;
    p->slots = slots;
    p->n_tiles = n_tiles;
    if (p->graph_exec) {
        cudaGraphExecDestroy(p->graph_exec);
        p->graph_exec = nullptr;
    }
    return cudaSuccess;
}

namespace {

cudaError_t build_batched_meta(art_portfolio* p) {
    const int L = p->n_layers;
    const int np = p->pool_np;
    cudaError_t e;
    if ((e = cudaMalloc(&p->d_elt_terms, sizeof(float) * 3 * np))) return e;
    if ((e = cudaMalloc(&p->d_elt_terms64, sizeof(double) * 3 * np))) return e;
    if ((e = cudaMalloc(&p->d_occ, sizeof(float) * 2 * L))) return e;
    if ((e = cudaMalloc(&p->d_agg, sizeof(double) * 2 * L))) return e;
    if ((e = cudaMalloc(&p->d_work_counter, sizeof(unsigned int)))) return e;
    if ((e = set_layer_tile(p, L <= 64 ? 2 : (L <= 128 ? 4 : 8)))) return e;
    return upload_batched_terms(p);
}

// Layer groups for the bitmap-skip kernel: consecutive layers while the
// group has at most 8 layers and the union of their ELTs at most 32.
void form_groups(art_portfolio* p) {
    p->group_elts.clear();
    p->group_layers.clear();
    std::vector<int32_t> uni, lay;
    for (int32_t j = 0; j < p->n_layers; ++j) {
        std::vector<int32_t> merged = uni;
        for (int c = p->loff[j]; c < p->loff[j + 1]; ++c)
            if (std::find(merged.begin(), merged.end(), p->lids[c]) == merged.end()) merged.push_back(p->lids[c]);
        if (!lay.empty() && ((int)lay.size() >= kMaxGroupLayers || (int)merged.size() > kMaxLayerElts)) {
            p->group_elts.push_back(uni);
            p->group_layers.push_back(lay);
            uni.clear();
            lay.clear();
            merged.clear();
            for (int c = p->loff[j]; c < p->loff[j + 1]; ++c) merged.push_back(p->lids[c]);
        }
        uni = merged;
        lay.push_back(j);
    }
    if (!lay.empty()) {
        p->group_elts.push_back(uni);
        p->group_layers.push_back(lay);
    }
}

// Terms of every group as its kernel reads them (kernel parameters).
void refresh_group_terms(art_portfolio* p) {
    for (size_t gi = 0; gi < p->groups.size(); ++gi) {
        GroupArgs& g = p->groups[gi];
        const std::vector<int32_t>& el = p->group_elts[gi];
        const std::vector<int32_t>& ly = p->group_layers[gi];
        for (int k = 0; k < kMaxLayerElts; ++k) {
            const bool real = k < (int)el.size();
            g.m[k] = real ? p->mult[el[k]] : 1.0f;
            g.d[k] = real ? p->ded[el[k]] : 0.0f;
            g.lim[k] = real ? p->lim[el[k]] : std::numeric_limits<float>::infinity();
        }
        g.n_layers = (int32_t)ly.size();
        for (int s = 0; s < kMaxGroupLayers; ++s) {
            const bool real = s < (int)ly.size();
            const int32_t j = real ? ly[s] : 0;
            uint32_t mem = 0;
            if (real)
                for (int c = p->loff[j]; c < p->loff[j + 1]; ++c)
                    mem |= 1u << (std::find(el.begin(), el.end(), p->lids[c]) - el.begin());
            g.member[s] = mem;
            for (int k = 0; k < kMaxLayerElts; ++k) g.coef[s][k] = ((mem >> k) & 1u) ? 1.0f : 0.0f;
            g.occ_ret[s] = real ? p->occ_ret[j] : 0.0f;
            g.occ_lim[s] = real ? p->occ_lim[j] : 0.0f;
            g.agg_ret[s] = real ? p->agg_ret[j] : 0.0;
            g.agg_lim[s] = real ? p->agg_lim[j] : 0.0;
            g.layer[s] = real ? j : 0;
        }
    }
}

// Terms of every layer as the occurrence-table build reads them, and the
// aggregate terms of the occurrence groups (kernel parameters).
cudaError_t upload_layer_build(art_portfolio* p) {
    std::vector<LayerBuildArgs> lb(p->n_layers);
    for (int32_t j = 0; j < p->n_layers; ++j) {
        LayerBuildArgs& a = lb[j];
        a.table = p->layer_tab[j];
        const int32_t b = p->loff[j], n = p->loff[j + 1] - b;
        for (int k = 0; k < kMaxLayerElts; ++k) {
            const bool real = k < n;
            const int32_t e = real ? p->lids[b + k] : 0;
            a.m[k] = real ? p->mult[e] : 1.0f;
            a.d[k] = real ? p->ded[e] : 0.0f;
            a.lim[k] = real ? p->lim[e] : std::numeric_limits<float>::infinity();
        }
        a.occ_ret = p->occ_ret[j];
        a.occ_lim = p->occ_lim[j];
        a.np = p->layer_np[j];
        a.pad_ = 0;
    }
    for (std::vector<OccGroupArgs>* v : {&p->ogroups, &p->ogroups64})
        for (OccGroupArgs& g : *v)
            for (int s = 0; s < g.n_layers; ++s) {
                g.agg_ret[s] = p->agg_ret[g.layer[s]];
                g.agg_lim[s] = p->agg_lim[g.layer[s]];
            }
    return cudaMemcpy(p->d_lbuild, lb.data(), sizeof(LayerBuildArgs) * lb.size(), cudaMemcpyHostToDevice);
}

// Occurrence groups of the skip variant: runs of up to 8 consecutive layers,
// each with an occurrence-loss table [C][og_lp] and a zero-padded bitmap.
cudaError_t build_occ_groups(art_portfolio* p) {
    const int32_t L = p->n_layers;
    const int32_t per = std::min(L, kMaxOccLayers);
    p->og_lp = per <= 1 ? 1 : per <= 2 ? 2 : per <= 4 ? 4 : 8;
    const int32_t ng = (L + kMaxOccLayers - 1) / kMaxOccLayers;
    p->ogroups.assign(ng, OccGroupArgs{});
    p->og_occ.assign(ng, nullptr);
    p->og_bits.assign(ng, nullptr);
    std::vector<OccBuildGroup> bg(ng);
    // X has one more row than the catalogue and the bitmap one more bit (the
    // sentinel C, where out-of-range ids land: bit clear, row zero); the
    // bitmap is zero-padded to whole 16-byte groups (the trial pass copies it
    // into shared memory 16 bytes at a time)
    const size_t xb = sizeof(float) * ((size_t)p->catalogue + 1) * p->og_lp;
    const size_t bb = 16 * (((size_t)p->catalogue / 32 + 1 + 3) / 4);
    cudaError_t e = cudaSuccess;
    for (int32_t gi = 0; gi < ng && !e; ++gi) {
        if ((e = cudaMalloc(&p->og_occ[gi], xb))) break;
        if ((e = cudaMalloc(&p->og_bits[gi], bb))) break;
        if ((e = cudaMemset(p->og_occ[gi], 0, xb))) break;
        if ((e = cudaMemset(p->og_bits[gi], 0, bb))) break;
        p->occ_bytes += (int64_t)(xb + bb);
        OccGroupArgs& g = p->ogroups[gi];
        g.occ = p->og_occ[gi];
        g.occ_bits = p->og_bits[gi];
        g.n_layers = std::min(kMaxOccLayers, L - gi * kMaxOccLayers);
        bg[gi].occ = p->og_occ[gi];
        bg[gi].occ_bits = p->og_bits[gi];
        bg[gi].n_layers = g.n_layers;
        for (int s = 0; s < kMaxOccLayers; ++s) {
            const bool real = s < g.n_layers;
            g.layer[s] = real ? gi * kMaxOccLayers + s : 0;
            bg[gi].layer[s] = g.layer[s];
        }
    }
    if (e) return e;
    // the tables X are built from the CSR of the non-zero losses where it
    // exists: each event's entries come in ELT id order, so a layer that
    // lists its ELTs in ascending order sums them in its own order (the
    // absent zeros add exactly 0); for a layer listed out of order the build
    // re-sums the events with three or more of its entries from its
    // per-layer row (one or two terms give the same bits in any order)
    for (int32_t gi = 0; gi < ng; ++gi)
        for (int s = 0; s < p->ogroups[gi].n_layers; ++s) {
            const int32_t j = p->ogroups[gi].layer[s];
            for (int32_t c = p->loff[j] + 1; c < p->loff[j + 1]; ++c)
                if (!(p->lids[c - 1] < p->lids[c])) bg[gi].unsorted |= 1 << s;
        }
    if (p->pool_np > 0 && p->sp_ptr) {
        std::vector<uint8_t> sm((size_t)ng * p->pool_np, 0);
        for (int32_t gi = 0; gi < ng; ++gi)
            for (int s = 0; s < p->ogroups[gi].n_layers; ++s) {
                const int32_t j = p->ogroups[gi].layer[s];
                for (int c = p->loff[j]; c < p->loff[j + 1]; ++c)
                    sm[(size_t)gi * p->pool_np + p->lids[c]] |= (uint8_t)(1u << s);
            }
        if ((e = cudaMalloc(&p->d_slotmask, sm.size()))) return e;
        if ((e = cudaMemcpy(p->d_slotmask, sm.data(), sm.size(), cudaMemcpyHostToDevice))) return e;
    }
    if ((e = cudaMalloc(&p->d_lbuild, sizeof(LayerBuildArgs) * L))) return e;
    if ((e = cudaMalloc(&p->d_ogroups, sizeof(OccBuildGroup) * ng))) return e;
    if ((e = cudaMemcpy(p->d_ogroups, bg.data(), sizeof(OccBuildGroup) * ng, cudaMemcpyHostToDevice))) return e;
    if (p->layouts & ART_LAYOUT_OCC64) {
        // FP64 groups hold up to 4 layers, so that one group's table
        // ([C + 1][4] FP64: 64 MB for 2M events) stays in L2 during its pass
        const int32_t per64 = std::min(L, kMaxOcc64Layers);
        p->og_lp64 = per64 <= 1 ? 1 : per64 <= 2 ? 2 : 4;
        const int32_t ng64 = (L + kMaxOcc64Layers - 1) / kMaxOcc64Layers;
        const size_t xb64 = sizeof(double) * ((size_t)p->catalogue + 1) * p->og_lp64;
        p->ogroups64.assign(ng64, OccGroupArgs{});
        p->og_occ64.assign(ng64, nullptr);
        p->og_bits64.assign(ng64, nullptr);
        std::vector<OccBuildGroup> bg64(ng64);
        for (int32_t gi = 0; gi < ng64 && !e; ++gi) {
            if ((e = cudaMalloc(&p->og_occ64[gi], xb64))) break;
            if ((e = cudaMalloc(&p->og_bits64[gi], bb))) break;
            if ((e = cudaMemset(p->og_occ64[gi], 0, xb64))) break;
            if ((e = cudaMemset(p->og_bits64[gi], 0, bb))) break;
            p->occ64_bytes += (int64_t)(xb64 + bb);
            OccGroupArgs& g = p->ogroups64[gi];
            g.occ64 = p->og_occ64[gi];
            g.occ_bits = p->og_bits64[gi];
            g.n_layers = std::min(kMaxOcc64Layers, L - gi * kMaxOcc64Layers);
            bg64[gi].occ_bits = p->og_bits64[gi];
            bg64[gi].n_layers = g.n_layers;
            for (int s = 0; s < kMaxOccLayers; ++s) {
                const bool real = s < g.n_layers;
                g.layer[s] = real ? gi * kMaxOcc64Layers + s : 0;
                bg64[gi].layer[s] = g.layer[s];
            }
        }
        if (e) return e;
        if ((e = cudaMalloc(&p->d_occ64_max, sizeof(unsigned long long) * ng64))) return e;
        if ((e = cudaMemset(p->d_occ64_max, 0, sizeof(unsigned long long) * ng64))) return e;
        for (int32_t gi = 0; gi < ng64; ++gi) {
            p->ogroups64[gi].maxkey = p->d_occ64_max + gi;
            bg64[gi].maxkey = p->d_occ64_max + gi;
        }
        if (p->pool_np > 0) {  // slots of each FP64 group holding each pool ELT (for the CSR build)
            std::vector<uint8_t> sm((size_t)ng64 * p->pool_np, 0);
            for (int32_t gi = 0; gi < ng64; ++gi)
                for (int s = 0; s < p->ogroups64[gi].n_layers; ++s) {
                    const int32_t j = p->ogroups64[gi].layer[s];
                    for (int c = p->loff[j]; c < p->loff[j + 1]; ++c)
                        sm[(size_t)gi * p->pool_np + p->lids[c]] |= (uint8_t)(1u << s);
                }
            if ((e = cudaMalloc(&p->d_slotmask64, sm.size()))) return e;
            if ((e = cudaMemcpy(p->d_slotmask64, sm.data(), sm.size(), cudaMemcpyHostToDevice))) return e;
        }
        if ((e = cudaMalloc(&p->d_ogroups64, sizeof(OccBuildGroup) * ng64))) return e;
        if ((e = cudaMemcpy(p->d_ogroups64, bg64.data(), sizeof(OccBuildGroup) * ng64, cudaMemcpyHostToDevice))) return e;
        if ((e = cudaMalloc(&p->d_occ64_ptrs, sizeof(double*) * ng64))) return e;
        if ((e = cudaMemcpy(p->d_occ64_ptrs, p->og_occ64.data(), sizeof(double*) * ng64, cudaMemcpyHostToDevice)))
            return e;
    }
    return upload_layer_build(p);
}

cudaError_t build_groups(art_portfolio* p, const float* losses, cudaStream_t stream) {
    form_groups(p);
    const size_t ng = p->group_elts.size();
    p->groups.assign(ng, GroupArgs{});
    p->group_np.assign(ng, 0);
    p->group_tab.assign(ng, nullptr);
    p->group_bitmap.assign(ng, nullptr);
    int32_t* d_el = nullptr;
    cudaError_t e = cudaMalloc(&d_el, sizeof(int32_t) * kMaxLayerElts * ng);
    if (e) return e;
    for (size_t gi = 0; gi < ng && !e; ++gi) {
        const std::vector<int32_t>& el = p->group_elts[gi];
        const int np = pad_np((int)el.size());
        p->group_np[gi] = np;
        const size_t tb = sizeof(float) * (size_t)p->catalogue * np;
        const size_t bb = sizeof(uint32_t) * (((size_t)p->catalogue + 31) / 32);
        if ((e = cudaMalloc(&p->group_tab[gi], tb))) break;
        if ((e = cudaMalloc(&p->group_bitmap[gi], bb))) break;
        p->group_bytes += (int64_t)(tb + bb);
        if ((e = cudaMemcpyAsync(d_el + gi * kMaxLayerElts, el.data(), sizeof(int32_t) * el.size(),
                                 cudaMemcpyHostToDevice, stream)))
            break;
        if ((e = build_layer_table(losses, p->catalogue, d_el + gi * kMaxLayerElts, (int32_t)el.size(), np,
                                   p->group_tab[gi], stream)))
            break;
        if ((e = build_group_bitmap(p->group_tab[gi], p->catalogue, np, p->group_bitmap[gi], stream))) break;
        p->groups[gi].table = p->group_tab[gi];
        p->groups[gi].bitmap = p->group_bitmap[gi];
    }
    const cudaError_t e2 = cudaStreamSynchronize(stream);
    cudaFree(d_el);
    if (e) return e;
    if (e2) return e2;
    refresh_group_terms(p);
    return cudaSuccess;
}

// Shared memory of the sparse kernel: ELT terms, the tiles' scatter lists and
// one [32 events][32 * slots + 1] FP32 accumulator block per warp.
size_t sparse_smem(const art_portfolio* p, int warps) {
    const size_t terms = (size_t)p->pool_np * 16;
    const size_t off = (((size_t)p->n_tiles * (p->pool_np + 1) * 2) + 15) & ~(size_t)15;
    const size_t lay = (size_t)p->n_tiles * p->tl_stride;
    const size_t x = (size_t)warps * 32 * (32 * p->slots + 1) * 4;
    return terms + off + lay + x;
}

size_t batched_smem(const art_portfolio* p, bool fp64) {
    return 3 * (size_t)p->pool_np * (fp64 ? 8 : 4) + (size_t)p->n_tiles * p->pool_np * 32;
}

void free_portfolio(art_portfolio* p) {
    if (!p) return;
    cudaDeviceSynchronize();
    for (float* t : p->layer_tab) cudaFree(t);
    for (float* t : p->group_tab) cudaFree(t);
    for (uint32_t* b : p->group_bitmap) cudaFree(b);
    for (float* t : p->og_occ) cudaFree(t);
    for (uint32_t* b : p->og_bits) cudaFree(b);
    cudaFree(p->d_lbuild);
    cudaFree(p->d_ogroups);
    for (double* t : p->og_occ64) cudaFree(t);
    for (uint32_t* b : p->og_bits64) cudaFree(b);
    cudaFree(p->d_ogroups64);
    cudaFree(p->d_occ64_ptrs);
    cudaFree(p->d_occ64_max);
    cudaFree(p->d_slotmask);
    cudaFree(p->d_slotmask64);
    cudaFree(p->pool);
    cudaFree(p->pool64);
    cudaFree(p->d_elt_terms);
    cudaFree(p->d_elt_terms64);
    cudaFree(p->d_memb);
    cudaFree(p->d_slot_layer);
    cudaFree(p->d_occ);
    cudaFree(p->d_agg);
    cudaFree(p->d_work_counter);
    cudaFree(p->sp_ptr);
    cudaFree(p->sp_entries);
    cudaFree(p->d_tl_off);
    cudaFree(p->d_tl_lay);
    cudaFree(p->d_flags);
    cudaFree(p->d_loff);
    cudaFree(p->d_lids);
    for (int i = 0; i < 2; ++i) {
        cudaFree(p->stage_ids[i]);
        cudaFree(p->stage_off[i]);
        cudaFree(p->stage_ylt[i]);
        if (p->ev_copied[i]) cudaEventDestroy(p->ev_copied[i]);
        if (p->ev_done[i]) cudaEventDestroy(p->ev_done[i]);
    }
    cudaFree(p->host_ylt);
    cudaFree(p->host_out);
    cudaFree(p->host_scratch);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    delete p;
}

int resolve_variant(const art_portfolio* p) {
    if (p->variant != ART_VARIANT_AUTO) return p->variant;
    // few groups: the YET is streamed once per group, each event row read
    // only when its bit is set; many groups: one pass over a pool table
    if (!p->groups.empty() && p->groups.size() <= 2) return ART_VARIANT_SKIP;
    if (p->sp_ptr && p->n_tiles > 0) return ART_VARIANT_SPARSE;
    if (p->pool && p->n_tiles > 0) return ART_VARIANT_BATCHED;
    if (!p->groups.empty()) return ART_VARIANT_SKIP;
    return ART_VARIANT_PLAIN;
}

bool variant_available(const art_portfolio* p, int v) {
    if (v == ART_VARIANT_PLAIN) return (p->layouts & ART_LAYOUT_LAYER) != 0;
    if (v == ART_VARIANT_SKIP) return !p->ogroups.empty();
    if (v == ART_VARIANT_SPARSE) return p->sp_ptr != nullptr && p->n_tiles > 0 && sparse_smem(p, 1) <= 200 * 1024;
    if (v == ART_VARIANT_BATCHED) return p->pool != nullptr && p->n_tiles > 0 && batched_smem(p, false) <= 200 * 1024;
    if (v == ART_VARIANT_FP64)
        return !p->ogroups64.empty() ||
               (p->pool64 != nullptr && p->n_tiles > 0 && batched_smem(p, true) <= 200 * 1024);
    return false;
}

art_status validate_yet(int64_t n_trials, const int32_t* ids, const int64_t* off, int32_t k) {
    if (n_trials < 0 || n_trials > (int64_t)1 << 40) return ART_EINVAL;
    if (!off && k < 0) return ART_EINVAL;
    if (!off && n_trials > 0 && k > 0 && n_trials > ((int64_t)1 << 62) / k) return ART_EINVAL;
    if (n_trials > 0 && !ids && (off || k > 0)) return ART_EINVAL;
    return ART_OK;
}

// build_tables false: the skip and all-FP64 variants reuse the occurrence
// tables a previous call on the stream wrote (the host-run path builds them
// once for all its chunks).
cudaError_t run_forward(art_portfolio* p, int variant, const YetArgs& y, double* ylt, uint8_t* branch,
                        cudaStream_t s, bool build_tables = true) {
    if (variant == ART_VARIANT_PLAIN) return launch_plain(p, y, ylt, branch, s);
    if (variant == ART_VARIANT_SKIP) return launch_skip(p, y, ylt, branch, s, build_tables);
    if (variant == ART_VARIANT_SPARSE) return launch_sparse(p, y, ylt, branch, s);
    if (variant == ART_VARIANT_FP64 && !p->ogroups64.empty()) return launch_skip64(p, y, ylt, branch, s, build_tables);
    return launch_batched(p, y, ylt, branch, variant == ART_VARIANT_FP64, s);
}

}  // namespace

extern "C" {

const char* art_status_string(art_status s) {
    switch (s) {
        case ART_OK: return "ART_OK";
        case ART_EINVAL: return "ART_EINVAL: invalid argument";
        case ART_ENOMEM: return "ART_ENOMEM: device allocation failed";
        case ART_ECUDA: return "ART_ECUDA: CUDA runtime error";
        case ART_EID_RANGE: return "ART_EID_RANGE: event id outside the catalogue";
        case ART_ETIMEOUT: return "ART_ETIMEOUT: bounded wait gave up";
        case ART_EUNSUPPORTED: return "ART_EUNSUPPORTED: layout not built for this call";
    }
    return "unknown art_status";
}

const char* art_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

int32_t art_version(void) { return 10000; }

art_status art_create_portfolio(int32_t catalogue_size, int32_t n_elt, const float* elt_losses_dev,
                                const float* elt_mult_host, const float* elt_ded_host, const float* elt_lim_host,
                                int32_t n_layers, const int32_t* layer_elt_off_host,
                                const int32_t* layer_elt_ids_host, const art_layer_terms* terms_host,
                                const art_options* opt, cudaStream_t stream, art_portfolio** out) {
    if (!out) return ART_EINVAL;
    *out = nullptr;
    if (catalogue_size < 1 || n_elt < 1 || n_elt > 4096 || n_layers < 1 || n_layers > 65536) return ART_EINVAL;
    if (!elt_losses_dev || !elt_ded_host || !elt_lim_host || !layer_elt_off_host || !layer_elt_ids_host ||
        !terms_host)
        return ART_EINVAL;
    if (layer_elt_off_host[0] != 0) return ART_EINVAL;
    for (int32_t j = 0; j < n_layers; ++j) {
        const int32_t b = layer_elt_off_host[j], e = layer_elt_off_host[j + 1];
        if (e - b < 1 || e - b > kMaxLayerElts) return ART_EINVAL;
        for (int32_t c = b; c < e; ++c) {
            const int32_t id = layer_elt_ids_host[c];
            if (id < 0 || id >= n_elt) return ART_EINVAL;
            for (int32_t c2 = b; c2 < c; ++c2)
                if (layer_elt_ids_host[c2] == id) return ART_EINVAL;
        }
    }
    auto* p = new art_portfolio();
    p->catalogue = catalogue_size;
    p->n_elt = n_elt;
    p->n_layers = n_layers;
    std::vector<float> ones(n_elt, 1.0f);
    if (!round_terms(n_elt, elt_mult_host ? elt_mult_host : ones.data(), elt_ded_host, elt_lim_host, n_layers,
                     terms_host, p->mult, p->ded, p->lim, p->occ_ret, p->occ_lim, p->agg_ret, p->agg_lim)) {
        delete p;
        return ART_EINVAL;
    }
    p->loff.assign(layer_elt_off_host, layer_elt_off_host + n_layers + 1);
    p->lids.assign(layer_elt_ids_host, layer_elt_ids_host + p->loff.back());
    p->layouts = (opt && opt->layouts) ? opt->layouts
                                       : (ART_LAYOUT_LAYER | ART_LAYOUT_POOL | ART_LAYOUT_GROUP | ART_LAYOUT_SPARSE);
    p->variant = opt ? opt->variant : ART_VARIANT_AUTO;
    p->flags = opt ? opt->flags : 0;
    p->trial_tile = opt ? opt->trial_tile : 0;
    p->cta_threads = opt ? opt->cta_threads : 0;
    if (p->variant < ART_VARIANT_AUTO || p->variant > ART_VARIANT_SPARSE || p->trial_tile < 0 ||
        (p->cta_threads != 0 && (p->cta_threads % 32 != 0 || p->cta_threads > 1024))) {
        delete p;
        return ART_EINVAL;
    }

    cudaError_t e;
    art_status st = ART_OK;
    do {
        if ((e = cudaGetDevice(&p->device))) break;
        if ((e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device))) break;
        if ((e = cudaMalloc(&p->d_flags, sizeof(int) * kNumFlags))) break;
        if ((e = cudaMemsetAsync(p->d_flags, 0, sizeof(int) * kNumFlags, stream))) break;
        // losses must be finite and >= 0 (zero where an ELT has no loss)
        const int64_t n_vals = (int64_t)n_elt * catalogue_size;
        check_losses_kernel<<<(unsigned)std::min<int64_t>((n_vals + 255) / 256, 4096), 256, 0, stream>>>(
            elt_losses_dev, n_vals, p->d_flags);
        if ((e = cudaGetLastError())) break;
        int bad = 0;
        if ((e = cudaMemcpyAsync(&bad, p->d_flags, sizeof(int), cudaMemcpyDeviceToHost, stream))) break;
        if ((e = cudaStreamSynchronize(stream))) break;
        if (bad) {
            st = ART_EINVAL;
            break;
        }
        if ((e = cudaMalloc(&p->d_loff, sizeof(int32_t) * p->loff.size()))) break;
        if ((e = cudaMalloc(&p->d_lids, sizeof(int32_t) * p->lids.size()))) break;
        if ((e = cudaMemcpy(p->d_loff, p->loff.data(), sizeof(int32_t) * p->loff.size(), cudaMemcpyHostToDevice))) break;
        if ((e = cudaMemcpy(p->d_lids, p->lids.data(), sizeof(int32_t) * p->lids.size(), cudaMemcpyHostToDevice))) break;
        if (p->layouts & ART_LAYOUT_LAYER) {
            p->layer_tab.assign(n_layers, nullptr);
            p->layer_np.assign(n_layers, 0);
            for (int32_t j = 0; j < n_layers && !e; ++j) {
                const int32_t n = p->loff[j + 1] - p->loff[j];
                const int32_t np = pad_np(n);
                p->layer_np[j] = np;
                const size_t bytes = sizeof(float) * (size_t)catalogue_size * np;
                if ((e = cudaMalloc(&p->layer_tab[j], bytes))) break;
                p->layer_bytes += (int64_t)bytes;
                e = build_layer_table(elt_losses_dev, catalogue_size, p->d_lids + p->loff[j], n, np, p->layer_tab[j],
                                      stream);
            }
            if (e) break;
        }
        if ((p->layouts & (ART_LAYOUT_POOL | ART_LAYOUT_POOL64 | ART_LAYOUT_SPARSE)) && n_elt <= kMaxPoolElts) {
            int epl = 1;
            while (32 * epl < n_elt) epl *= 2;
            p->pool_np = 32 * epl;
            if (p->layouts & ART_LAYOUT_POOL) {
                const size_t bytes = sizeof(float) * (size_t)catalogue_size * p->pool_np;
                if ((e = cudaMalloc(&p->pool, bytes))) break;
                p->pool_bytes = (int64_t)bytes;
            }
            if (p->layouts & ART_LAYOUT_POOL64) {
                const size_t bytes = sizeof(double) * (size_t)catalogue_size * p->pool_np;
                if ((e = cudaMalloc(&p->pool64, bytes))) break;
                p->pool64_bytes = (int64_t)bytes;
            }
            if ((p->pool || p->pool64) &&
                (e = build_pool_table(elt_losses_dev, catalogue_size, n_elt, p->pool_np, p->pool, p->pool64, stream)))
                break;
            if ((e = build_batched_meta(p))) break;
            // the CSR offsets are 32-bit: build it when every count fits
            if ((p->layouts & ART_LAYOUT_SPARSE) && (int64_t)n_elt * catalogue_size < ((int64_t)1 << 32) &&
                (e = build_sparse(p, elt_losses_dev, stream)))
                break;
        }
        // occurrence groups of the skip (and all-FP64) variants, after the
        // pool width is known (the FP64 tables' CSR build masks span it)
        if ((p->layouts & ART_LAYOUT_LAYER) && (e = build_occ_groups(p))) break;
        if ((p->layouts & ART_LAYOUT_GROUP) && (e = build_groups(p, elt_losses_dev, stream))) break;
        if (p->flags & ART_FLAG_L2_PERSIST) {
            int persist_max = 0;
            cudaDeviceGetAttribute(&persist_max, cudaDevAttrMaxPersistingL2CacheSize, p->device);
            if (persist_max > 0 && (e = cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)persist_max))) break;
        }
        e = cudaStreamSynchronize(stream);
    } while (0);
    if (e != cudaSuccess || st != ART_OK) {
        const art_status r = e != cudaSuccess ? fail(e) : st;
        free_portfolio(p);
        return r;
    }
    if (p->variant != ART_VARIANT_AUTO && !variant_available(p, p->variant)) {
        free_portfolio(p);
        return ART_EUNSUPPORTED;
    }
    *out = p;
    return ART_OK;
}

art_status art_update_terms(art_portfolio* p, const float* elt_mult_host, const float* elt_ded_host,
                            const float* elt_lim_host, const art_layer_terms* terms_host) {
    if (!p) return ART_EINVAL;
    std::vector<float> m = p->mult, d = p->ded, l = p->lim, orr = p->occ_ret, orl = p->occ_lim;
    std::vector<double> oar = p->agg_ret, oal = p->agg_lim;
    if (!round_terms(p->n_elt, elt_mult_host, elt_ded_host, elt_lim_host, p->n_layers, terms_host, m, d, l, orr, orl,
                     oar, oal))
        return ART_EINVAL;
    p->mult.swap(m);
    p->ded.swap(d);
    p->lim.swap(l);
    p->occ_ret.swap(orr);
    p->occ_lim.swap(orl);
    p->agg_ret.swap(oar);
    p->agg_lim.swap(oal);
    if (p->d_elt_terms) {
        const cudaError_t e = upload_batched_terms(p);
        if (e) return fail(e);
    }
    refresh_group_terms(p);
    if (p->d_lbuild) {
        const cudaError_t e = upload_layer_build(p);
        if (e) return fail(e);
    }
    if (p->graph_exec) {  // the plain variant bakes terms into launch parameters
        cudaGraphExecDestroy(p->graph_exec);
        p->graph_exec = nullptr;
    }
    return ART_OK;
}

art_status art_get_terms(const art_portfolio* p, float* elt_mult_host, float* elt_ded_host, float* elt_lim_host,
                         art_layer_terms* terms_host) {
    if (!p) return ART_EINVAL;
    if (elt_mult_host) std::copy(p->mult.begin(), p->mult.end(), elt_mult_host);
    if (elt_ded_host) std::copy(p->ded.begin(), p->ded.end(), elt_ded_host);
    if (elt_lim_host) std::copy(p->lim.begin(), p->lim.end(), elt_lim_host);
    if (terms_host)
        for (int32_t j = 0; j < p->n_layers; ++j)
            terms_host[j] = art_layer_terms{p->occ_ret[j], p->occ_lim[j], p->agg_ret[j], p->agg_lim[j]};
    return ART_OK;
}

art_status art_set_flags(art_portfolio* p, int32_t flags) {
    if (!p || (flags & ~(ART_FLAG_L2_PERSIST | ART_FLAG_GRAPH | ART_FLAG_EARLY_EXIT | ART_FLAG_HOST_STAGED)))
        return ART_EINVAL;
    p->flags = flags;
    if (p->graph_exec) {
        cudaGraphExecDestroy(p->graph_exec);
        p->graph_exec = nullptr;
    }
    return ART_OK;
}

art_status art_set_variant(art_portfolio* p, int32_t variant, int32_t trial_tile, int32_t cta_threads) {
    if (!p || variant < ART_VARIANT_AUTO || variant > ART_VARIANT_SPARSE || trial_tile < 0 || cta_threads < 0 ||
        cta_threads % 32 != 0 || cta_threads > 1024)
        return ART_EINVAL;
    if (variant != ART_VARIANT_AUTO && !variant_available(p, variant)) return ART_EUNSUPPORTED;
    p->variant = variant;
    if (trial_tile) p->trial_tile = trial_tile;
    if (cta_threads) p->cta_threads = cta_threads;
    if (p->graph_exec) {
        cudaGraphExecDestroy(p->graph_exec);
        p->graph_exec = nullptr;
    }
    return ART_OK;
}

art_status art_run_ylt(art_portfolio* p, int64_t n_trials, const int32_t* event_ids_dev,
                       const int64_t* trial_off_dev, int32_t events_per_trial, double* ylt_dev, uint8_t* branch_dev,
                       cudaStream_t stream) {
    if (!p) return ART_EINVAL;
    art_status st = validate_yet(n_trials, event_ids_dev, trial_off_dev, events_per_trial);
    if (st) return st;
    if (n_trials == 0) return ART_OK;
    if (!ylt_dev) return ART_EINVAL;
    const int variant = resolve_variant(p);
    if (!variant_available(p, variant)) return ART_EUNSUPPORTED;
    YetArgs y{event_ids_dev, trial_off_dev, n_trials, trial_off_dev ? 0 : events_per_trial, p->catalogue};
    cudaError_t e;
    const bool use_graph = (p->flags & ART_FLAG_GRAPH) != 0;
    if (use_graph) {
        const void* key[4] = {event_ids_dev, trial_off_dev, ylt_dev, branch_dev};
        const bool hit = p->graph_exec && std::equal(key, key + 4, p->graph_key) && p->graph_key_n[0] == n_trials &&
                         p->graph_key_n[1] == ((int64_t)events_per_trial << 4 | variant);
        if (!hit) {
            if (p->graph_exec) {
                cudaGraphExecDestroy(p->graph_exec);
                p->graph_exec = nullptr;
            }
            cudaStream_t cap;
            if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking))) return fail(e);
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (!e) {
                const cudaError_t le = run_forward(p, variant, y, ylt_dev, branch_dev, cap);
                e = cudaStreamEndCapture(cap, &g);
                if (!e) e = le;
            }
            if (!e) e = cudaGraphInstantiate(&p->graph_exec, g, 0);
            if (g) cudaGraphDestroy(g);
            cudaStreamDestroy(cap);
            if (e) {
                p->graph_exec = nullptr;
                return fail(e);
            }
            std::copy(key, key + 4, p->graph_key);
            p->graph_key_n[0] = n_trials;
            p->graph_key_n[1] = ((int64_t)events_per_trial << 4 | variant);
        }
        e = cudaGraphLaunch(p->graph_exec, stream);
        return e ? fail(e) : ART_OK;
    }
    // the skip variant sets its own windows, one per occurrence group
    const bool window = (p->flags & ART_FLAG_L2_PERSIST) != 0 && variant != ART_VARIANT_PLAIN &&
                        variant != ART_VARIANT_SKIP;
    if (window) set_window(stream, variant == ART_VARIANT_FP64 ? (const void*)p->pool64 : (const void*)p->pool,
                           variant == ART_VARIANT_FP64 ? p->pool64_bytes : p->pool_bytes);
    e = run_forward(p, variant, y, ylt_dev, branch_dev, stream);
    if (window) set_window(stream, nullptr, 0);
    return e ? fail(e) : ART_OK;
}

}  // extern "C"

namespace {

// A device buffer of at least `need` doubles, kept by the portfolio between
// calls (reallocated, after the stream's work, only when it grows).
cudaError_t ensure_dev(double** buf, int64_t* cap, int64_t need, cudaStream_t stream) {
    if (need <= *cap) return cudaSuccess;
    cudaStreamSynchronize(stream);
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    const cudaError_t e = cudaMalloc(buf, sizeof(double) * (size_t)need);
    if (e == cudaSuccess) *cap = need;
    return e;
}

// The current device's address of a host buffer that is page-locked and
// mapped into it (cudaHostAlloc, cudaHostRegister with mapping, a pinned
// tensor under unified addressing); NULL for any other buffer (the failed
// query's error is cleared).
template <typename T>
const T* device_alias(const T* host) {
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, const_cast<T*>(host), 0) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return static_cast<const T*>(d);
}

// True when the variant's forward reads every event id once per call: the
// skip and all-FP64 variants with one occurrence group, the plain variant
// with one layer.
bool one_pass_over_ids(const art_portfolio* p, int variant) {
    if (variant == ART_VARIANT_SKIP) return p->ogroups.size() == 1;
    if (variant == ART_VARIANT_FP64) return p->ogroups64.size() == 1;
    if (variant == ART_VARIANT_PLAIN) return p->n_layers == 1;
    return false;
}

// The host-buffer forward. When the YET buffers are mapped page-locked host
// memory and the variant reads every id once, the forward reads them in
// place over the host link (no staging copies; ART_FLAG_HOST_STAGED turns
// this off) into ylt_dev, or a device YLT the portfolio keeps, and the YLT
// is copied to ylt_host. Otherwise the YET goes to the device in chunks of
// trials on `stream` (copies on the portfolio's copy stream,
// double-buffered), each chunk's YLT rows go to ylt_host (if not NULL) and
// into columns t0.. of the device array ylt_dev ([n_layers][n_trials], if
// not NULL). Blocks until the last copy is done. Arguments validated by the
// caller.
art_status host_run(art_portfolio* p, int64_t n_trials, const int32_t* event_ids_host, const int64_t* trial_off_host,
                    int32_t events_per_trial, double* ylt_host, double* ylt_dev, cudaStream_t stream) {
    if (trial_off_host) {
        if (trial_off_host[0] != 0) return ART_EINVAL;
        for (int64_t t = 0; t < n_trials; ++t)
            if (trial_off_host[t + 1] < trial_off_host[t]) return ART_EINVAL;
    }
    const int variant = resolve_variant(p);
    if (!variant_available(p, variant)) return ART_EUNSUPPORTED;
    if (!(p->flags & ART_FLAG_HOST_STAGED) && one_pass_over_ids(p, variant)) {
        const int32_t* d_ids = device_alias(event_ids_host);
        const int64_t* d_off = trial_off_host ? device_alias(trial_off_host) : nullptr;
        if (d_ids && (!trial_off_host || d_off)) {
            cudaError_t e = cudaSuccess;
            double* yd = ylt_dev;
            if (!yd) {
                if ((e = ensure_dev(&p->host_ylt, &p->host_ylt_cap, (int64_t)p->n_layers * n_trials, stream)))
                    return fail(e);
                yd = p->host_ylt;
            }
            const YetArgs y{d_ids, d_off, n_trials, trial_off_host ? 0 : events_per_trial, p->catalogue};
            e = run_forward(p, variant, y, yd, nullptr, stream, true);
            if (!e && ylt_host)
                e = cudaMemcpyAsync(ylt_host, yd, sizeof(double) * (size_t)p->n_layers * (size_t)n_trials,
                                    cudaMemcpyDeviceToHost, stream);
            const cudaError_t e2 = cudaStreamSynchronize(stream);
            if (e || e2) return fail(e ? e : e2);
            return ART_OK;
        }
    }
    // chunk of trials per stage: about 64 MiB of ids
    const int64_t avg = trial_off_host ? std::max<int64_t>(1, trial_off_host[n_trials] / std::max<int64_t>(1, n_trials))
                                       : std::max<int64_t>(1, events_per_trial);
    int64_t chunk = std::max<int64_t>(1024, ((int64_t)16 << 20) / avg);
    chunk = std::min(chunk, n_trials);
    // largest id span of any chunk
    int64_t max_ids = 0;
    for (int64_t t0 = 0; t0 < n_trials; t0 += chunk) {
        const int64_t t1 = std::min(n_trials, t0 + chunk);
        const int64_t span = trial_off_host ? trial_off_host[t1] - trial_off_host[t0] : (t1 - t0) * events_per_trial;
        max_ids = std::max(max_ids, span);
    }
    cudaError_t e = cudaSuccess;
    if (max_ids > p->stage_ids_cap || chunk > p->stage_trials_cap) {
        cudaStreamSynchronize(stream);
        for (int i = 0; i < 2; ++i) {
            cudaFree(p->stage_ids[i]);
            cudaFree(p->stage_off[i]);
            cudaFree(p->stage_ylt[i]);
            p->stage_ids[i] = nullptr;
            p->stage_off[i] = nullptr;
            p->stage_ylt[i] = nullptr;
        }
        p->stage_ids_cap = p->stage_trials_cap = 0;
        for (int i = 0; i < 2 && !e; ++i) {
            if ((e = cudaMalloc(&p->stage_ids[i], sizeof(int32_t) * std::max<int64_t>(1, max_ids)))) break;
            if ((e = cudaMalloc(&p->stage_off[i], sizeof(int64_t) * (chunk + 1)))) break;
            e = cudaMalloc(&p->stage_ylt[i], sizeof(double) * (size_t)chunk * p->n_layers);
        }
        if (e) return fail(e);
        p->stage_ids_cap = max_ids;
        p->stage_trials_cap = chunk;
    }
    if (!p->copy_stream) {
        if ((e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking))) return fail(e);
        for (int i = 0; i < 2 && !e; ++i) {
            if ((e = cudaEventCreateWithFlags(&p->ev_copied[i], cudaEventDisableTiming))) break;
            e = cudaEventCreateWithFlags(&p->ev_done[i], cudaEventDisableTiming);
        }
        if (e) return fail(e);
    }
    // the copy stream must not run ahead of work already queued on `stream`
    if ((e = cudaEventRecord(p->ev_done[0], stream))) return fail(e);
    if ((e = cudaEventRecord(p->ev_done[1], stream))) return fail(e);
    // the occurrence tables of the skip and all-FP64 variants depend on the
    // terms only: written once here, read by every chunk
    const bool tables = variant == ART_VARIANT_SKIP || (variant == ART_VARIANT_FP64 && !p->ogroups64.empty());
    if (tables) {
        const YetArgs none{nullptr, nullptr, 0, 0, p->catalogue};
        if ((e = run_forward(p, variant, none, nullptr, nullptr, stream, true))) return fail(e);
    }
    int64_t c = 0;
    for (int64_t t0 = 0; t0 < n_trials && !e; t0 += chunk, ++c) {
        const int slot = (int)(c & 1);
        const int64_t t1 = std::min(n_trials, t0 + chunk), nt = t1 - t0;
        const int64_t i0 = trial_off_host ? trial_off_host[t0] : t0 * events_per_trial;
        const int64_t i1 = trial_off_host ? trial_off_host[t1] : t1 * events_per_trial;
        if ((e = cudaStreamWaitEvent(p->copy_stream, p->ev_done[slot], 0))) break;
        if (i1 > i0 && (e = cudaMemcpyAsync(p->stage_ids[slot], event_ids_host + i0, sizeof(int32_t) * (i1 - i0),
                                            cudaMemcpyHostToDevice, p->copy_stream)))
            break;
        if (trial_off_host && (e = cudaMemcpyAsync(p->stage_off[slot], trial_off_host + t0, sizeof(int64_t) * (nt + 1),
                                                   cudaMemcpyHostToDevice, p->copy_stream)))
            break;
        if ((e = cudaEventRecord(p->ev_copied[slot], p->copy_stream))) break;
        if ((e = cudaStreamWaitEvent(stream, p->ev_copied[slot], 0))) break;
        // offsets stay absolute: the ids pointer is shifted so that ids[off[t]]
        // lands in the staging buffer
        YetArgs y{p->stage_ids[slot] - i0, trial_off_host ? p->stage_off[slot] : nullptr, nt,
                  trial_off_host ? 0 : events_per_trial, p->catalogue};
        if (!trial_off_host) y.ids = p->stage_ids[slot];
        if ((e = run_forward(p, variant, y, p->stage_ylt[slot], nullptr, stream, !tables))) break;
        if (ylt_dev && (e = cudaMemcpy2DAsync(ylt_dev + t0, sizeof(double) * n_trials, p->stage_ylt[slot],
                                              sizeof(double) * nt, sizeof(double) * nt, p->n_layers,
                                              cudaMemcpyDeviceToDevice, stream)))
            break;
        if (ylt_host && (e = cudaMemcpy2DAsync(ylt_host + t0, sizeof(double) * n_trials, p->stage_ylt[slot],
                                               sizeof(double) * nt, sizeof(double) * nt, p->n_layers,
                                               cudaMemcpyDeviceToHost, stream)))
            break;
        e = cudaEventRecord(p->ev_done[slot], stream);
    }
    const cudaError_t e2 = cudaStreamSynchronize(stream);
    if (e || e2) return fail(e ? e : e2);
    return ART_OK;
}

bool valid_probs(const double* probs, int32_t n_p) {
    if (!probs || n_p < 1 || n_p > kMaxProbs) return false;
    for (int q = 0; q < n_p; ++q)
        if (!(probs[q] > 0.0 && probs[q] < 1.0)) return false;
    return true;
}

}  // namespace

extern "C" {

art_status art_run_ylt_host(art_portfolio* p, int64_t n_trials, const int32_t* event_ids_host,
                            const int64_t* trial_off_host, int32_t events_per_trial, double* ylt_host,
                            cudaStream_t stream) {
    if (!p) return ART_EINVAL;
    art_status st = validate_yet(n_trials, event_ids_host, trial_off_host, events_per_trial);
    if (st) return st;
    if (n_trials == 0) return ART_OK;
    if (!ylt_host) return ART_EINVAL;
    return host_run(p, n_trials, event_ids_host, trial_off_host, events_per_trial, ylt_host, nullptr, stream);
}

art_status art_run_ylt_host_metrics(art_portfolio* p, int64_t n_trials, const int32_t* event_ids_host,
                                    const int64_t* trial_off_host, int32_t events_per_trial, double* ylt_host,
                                    const double* probs_host, int32_t n_p, double* mean_host, double* pml_host,
                                    double* tvar_host, cudaStream_t stream) {
    if (!p) return ART_EINVAL;
    art_status st = validate_yet(n_trials, event_ids_host, trial_off_host, events_per_trial);
    if (st) return st;
    if (n_trials < 1 || n_trials > 0x7fffffffLL || p->n_layers > 65535 || !valid_probs(probs_host, n_p))
        return ART_EINVAL;
    const int64_t L = p->n_layers;
    const int64_t need_ylt = L * n_trials, need_out = L * (1 + 2 * (int64_t)n_p);
    cudaError_t e = cudaSuccess;
    if ((e = ensure_dev(&p->host_ylt, &p->host_ylt_cap, need_ylt, stream))) return fail(e);
    if ((e = ensure_dev(&p->host_out, &p->host_out_cap, need_out, stream))) return fail(e);
    // the metrics' scratch too, so that repeated calls allocate nothing
    const size_t need_scratch = metrics_scratch_bytes(n_trials, (int32_t)L, n_p);
    if (need_scratch > p->host_scratch_cap) {
        cudaStreamSynchronize(stream);
        cudaFree(p->host_scratch);
        p->host_scratch = nullptr;
        p->host_scratch_cap = 0;
        if ((e = cudaMalloc(&p->host_scratch, need_scratch))) return fail(e);
        p->host_scratch_cap = need_scratch;
    }
    // chunks of the YET through the forward; the YLT stays on the device too
    st = host_run(p, n_trials, event_ids_host, trial_off_host, events_per_trial, ylt_host, p->host_ylt, stream);
    if (st) return st;
    double* d_mean = p->host_out;
    double* d_pml = d_mean + L;
    double* d_tvar = d_pml + L * n_p;
    if ((e = metrics_run(p->host_ylt, n_trials, (int32_t)L, probs_host, n_p, d_mean, d_pml, d_tvar, stream,
                         p->host_scratch, p->host_scratch_cap)))
        return fail(e);
    if (mean_host && (e = cudaMemcpyAsync(mean_host, d_mean, sizeof(double) * L, cudaMemcpyDeviceToHost, stream)))
        return fail(e);
    if (pml_host &&
        (e = cudaMemcpyAsync(pml_host, d_pml, sizeof(double) * L * n_p, cudaMemcpyDeviceToHost, stream)))
        return fail(e);
    if (tvar_host &&
        (e = cudaMemcpyAsync(tvar_host, d_tvar, sizeof(double) * L * n_p, cudaMemcpyDeviceToHost, stream)))
        return fail(e);
    if ((e = cudaStreamSynchronize(stream))) return fail(e);
    return ART_OK;
}

art_status art_run_payouts(art_portfolio* p, int32_t layer, int64_t n_trials, const int32_t* event_ids_dev,
                           const int64_t* trial_off_dev, int32_t events_per_trial, double* payouts_dev,
                           int32_t* exhaust_dev, double* ylt_dev, cudaStream_t stream) {
    if (!p || layer < 0 || layer >= p->n_layers) return ART_EINVAL;
    const art_status st = validate_yet(n_trials, event_ids_dev, trial_off_dev, events_per_trial);
    if (st) return st;
    if (!(p->layouts & ART_LAYOUT_LAYER)) return ART_EUNSUPPORTED;
    YetArgs y{event_ids_dev, trial_off_dev, n_trials, trial_off_dev ? 0 : events_per_trial, p->catalogue};
    const cudaError_t e = launch_payouts(p, layer, y, payouts_dev, exhaust_dev, ylt_dev, stream);
    return e ? fail(e) : ART_OK;
}

art_status art_metrics(const double* ylt_dev, int64_t n_trials, int32_t n_layers, const double* probs_host,
                       int32_t n_p, double* mean_dev, double* pml_dev, double* tvar_dev, cudaStream_t stream) {
    if (!ylt_dev || n_trials < 1 || n_trials > 0x7fffffffLL || n_layers < 1 || n_layers > 65535 || !probs_host ||
        n_p < 1 || n_p > kMaxProbs)
        return ART_EINVAL;
    for (int q = 0; q < n_p; ++q)
        if (!(probs_host[q] > 0.0 && probs_host[q] < 1.0)) return ART_EINVAL;
    const cudaError_t e = metrics_run(ylt_dev, n_trials, n_layers, probs_host, n_p, mean_dev, pml_dev, tvar_dev, stream);
    return e ? fail(e) : ART_OK;
}

art_status art_metrics_backward(const double* ylt_dev, int64_t n_trials, int32_t n_layers, const double* probs_host,
                                int32_t n_p, const double* pml_dev, const double* grad_mean_dev,
                                const double* grad_tvar_dev, double* grad_ylt_dev, cudaStream_t stream) {
    if (!ylt_dev || !grad_ylt_dev || n_trials < 1 || n_trials > 0x7fffffffLL || n_layers < 1 || n_layers > 65535 ||
        n_p < 0 || n_p > kMaxProbs)
        return ART_EINVAL;
    if (grad_tvar_dev && (!pml_dev || !probs_host || n_p < 1)) return ART_EINVAL;
    for (int q = 0; q < n_p && probs_host; ++q)
        if (!(probs_host[q] > 0.0 && probs_host[q] < 1.0)) return ART_EINVAL;
    const cudaError_t e = metrics_backward_run(ylt_dev, n_trials, n_layers, probs_host, n_p, pml_dev, grad_mean_dev,
                                               grad_tvar_dev, grad_ylt_dev, stream);
    return e ? fail(e) : ART_OK;
}

art_status art_run_ylt_backward(art_portfolio* p, int64_t n_trials, const int32_t* event_ids_dev,
                                const int64_t* trial_off_dev, int32_t events_per_trial, const uint8_t* branch_dev,
                                const double* grad_ylt_dev, double* grad_terms_dev, double* grad_mult_dev,
                                cudaStream_t stream) {
    if (!p) return ART_EINVAL;
    art_status st = validate_yet(n_trials, event_ids_dev, trial_off_dev, events_per_trial);
    if (st) return st;
    if (!grad_terms_dev || !grad_mult_dev || (n_trials > 0 && (!branch_dev || !grad_ylt_dev))) return ART_EINVAL;
    if (!(p->layouts & (ART_LAYOUT_GROUP | ART_LAYOUT_LAYER))) return ART_EUNSUPPORTED;
    YetArgs y{event_ids_dev, trial_off_dev, n_trials, trial_off_dev ? 0 : events_per_trial, p->catalogue};
    // one pass per layer group where the group tables exist, else one per layer
    const cudaError_t e =
        (p->layouts & ART_LAYOUT_GROUP)
            ? launch_adjoint_groups(p, y, branch_dev, grad_ylt_dev, grad_terms_dev, grad_mult_dev, stream)
            : launch_adjoint(p, y, branch_dev, grad_ylt_dev, grad_terms_dev, grad_mult_dev, stream);
    return e ? fail(e) : ART_OK;
}

art_status art_get_device_status(art_portfolio* p, cudaStream_t stream) {
    if (!p) return ART_EINVAL;
    int flags[kNumFlags] = {0, 0, 0, 0};
    cudaError_t e = cudaStreamSynchronize(stream);
    if (!e) e = cudaMemcpy(flags, p->d_flags, sizeof(flags), cudaMemcpyDeviceToHost);
    if (!e) e = cudaMemset(p->d_flags, 0, sizeof(flags));
    if (e) return fail(e);
    if (flags[kFlagIdRange]) return ART_EID_RANGE;
    if (flags[kFlagBadOffsets]) return ART_EINVAL;
    return ART_OK;
}

art_status art_get_footprint(const art_portfolio* p, int64_t* layer_bytes, int64_t* pool_bytes, int64_t* pool64_bytes,
                             int64_t* group_bytes, int64_t* sparse_bytes) {
    if (!p) return ART_EINVAL;
    if (sparse_bytes) *sparse_bytes = p->sparse_bytes;
    if (group_bytes) *group_bytes = p->group_bytes;
    if (layer_bytes) *layer_bytes = p->layer_bytes + p->occ_bytes;
    if (pool_bytes) *pool_bytes = p->pool_bytes;
    if (pool64_bytes) *pool64_bytes = p->pool64_bytes + p->occ64_bytes;
    return ART_OK;
}

void art_destroy_portfolio(art_portfolio* p) { free_portfolio(p); }

// ---------------------------------------------------------------- autotuner

namespace {

std::string tune_key(const art_portfolio* p, int64_t n_trials, int32_t k, bool csr) {
    cudaDeviceProp prop;
    std::memset(&prop, 0, sizeof(prop));
    cudaGetDeviceProperties(&prop, p->device);
    int64_t sum_elts = 0;
    for (int32_t j = 0; j < p->n_layers; ++j) sum_elts += p->loff[j + 1] - p->loff[j];
    // trials bucketed by powers of two: the best shape does not move with a few trials
    int lg = 0;
    while (((int64_t)1 << (lg + 1)) <= n_trials) ++lg;
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s|sm%d|C%d|E%d|L%d|S%lld|T2^%d|K%d|%s|lay%d", prop.name, prop.multiProcessorCount,
                  p->catalogue, p->n_elt, p->n_layers, (long long)sum_elts, lg, k, csr ? "csr" : "dense", p->layouts);
    return buf;
}

bool cache_lookup(const std::string& key, int32_t* v) {
    const char* path = std::getenv("ART_AUTOTUNE_CACHE");
    if (!path || !*path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool hit = false;
    while (std::fgets(line, sizeof(line), f)) {
        char* tab = std::strchr(line, '\t');
        if (!tab) continue;
        *tab = 0;
        int32_t a, b, c, d, m = -1;
        const int got = std::sscanf(tab + 1, "%d %d %d %d %d", &a, &b, &c, &d, &m);
        if (key == line && got >= 4) {
            v[0] = a; v[1] = b; v[2] = c; v[3] = d; v[4] = got == 5 ? m : -1;
            hit = true;  // the last matching line wins
        }
    }
    std::fclose(f);
    return hit;
}

void cache_store(const std::string& key, const int32_t* v, float ms) {
    const char* path = std::getenv("ART_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s\t%d %d %d %d %d\t%.4f\n", key.c_str(), v[0], v[1], v[2], v[3], v[4], ms);
    std::fclose(f);
}

cudaError_t apply_shape(art_portfolio* p, const int32_t* v) {
    if ((v[0] == ART_VARIANT_BATCHED || v[0] == ART_VARIANT_SPARSE || v[0] == ART_VARIANT_FP64) && v[1] != p->slots) {
        const cudaError_t e = set_layer_tile(p, v[1]);
        if (e) return e;
    }
    p->variant = v[0];
    p->trial_tile = v[2];
    p->cta_threads = v[3];
    p->sparse_mapping = v[4];
    if (p->graph_exec) {
        cudaGraphExecDestroy(p->graph_exec);
        p->graph_exec = nullptr;
    }
    return cudaSuccess;
}

}  // namespace

art_status art_autotune(art_portfolio* p, int64_t n_trials, const int32_t* event_ids_dev, const int64_t* trial_off_dev,
                        int32_t events_per_trial, double* ylt_dev, int32_t sample_trials, cudaStream_t stream,
                        art_tune_result* out) {
    if (!p || !ylt_dev || sample_trials < 0) return ART_EINVAL;
    art_status st = validate_yet(n_trials, event_ids_dev, trial_off_dev, events_per_trial);
    if (st) return st;
    if (n_trials < 1) return ART_EINVAL;
    const int64_t ts = std::min<int64_t>(n_trials, sample_trials > 0 ? sample_trials : 65536);
    YetArgs y{event_ids_dev, trial_off_dev, ts, trial_off_dev ? 0 : events_per_trial, p->catalogue};
    const std::string key = tune_key(p, n_trials, events_per_trial, trial_off_dev != nullptr);
    int32_t best[5] = {p->variant, p->slots, p->trial_tile, p->cta_threads, p->sparse_mapping};
    art_tune_result res;
    std::memset(&res, 0, sizeof(res));
    cudaError_t e = cudaSuccess;
    if (cache_lookup(key, best)) {
        const bool usable = variant_available(p, best[0]) || best[0] == ART_VARIANT_AUTO;
        if (usable) {
            if ((e = apply_shape(p, best))) return fail(e);
            res.variant = best[0]; res.slots = best[1]; res.trial_tile = best[2]; res.cta_threads = best[3];
            res.mapping = best[4];
            res.from_cache = 1;
            if (out) *out = res;
            return ART_OK;
        }
    }
    // candidates: (variant, slots, trial tile, CTA threads)
    std::vector<std::array<int32_t, 5>> cands;
    if (variant_available(p, ART_VARIANT_PLAIN)) cands.push_back({ART_VARIANT_PLAIN, p->slots, 0, 0, -1});
    if (variant_available(p, ART_VARIANT_SKIP)) cands.push_back({ART_VARIANT_SKIP, p->slots, 0, 0, -1});
    const int32_t slot_opts[3] = {2, 4, 8};
    for (int v : {ART_VARIANT_BATCHED, ART_VARIANT_SPARSE}) {
        if (!variant_available(p, v)) continue;
        for (int32_t sl : slot_opts) {
            const int per_tile = 32 * sl;
            const int64_t tiles = (p->n_layers + per_tile - 1) / per_tile;
            if (sl > 2 && 32 * (sl / 2) >= p->n_layers) continue;  // no fewer tiles than a smaller slot count
            if ((size_t)p->pool_np * 16 + (size_t)tiles * p->pool_np * 32 > 200 * 1024) continue;
            if (v == ART_VARIANT_SPARSE &&
                (size_t)p->pool_np * 18 + (size_t)tiles * (p->pool_np + 8192) + 32 * (32 * sl + 1) * 4 > 200 * 1024)
                continue;
            for (int32_t tt : {1, 2, 4, 8, 16})
                for (int32_t th : {128, 256}) {
                    if (v == ART_VARIANT_SPARSE) {
                        cands.push_back({v, sl, tt, th, 0});
                        cands.push_back({v, sl, tt, th, 1});
                    } else {
                        cands.push_back({v, sl, tt, th, -1});
                    }
                }
        }
    }
    const int32_t saved[5] = {p->variant, p->slots, p->trial_tile, p->cta_threads, p->sparse_mapping};
    cudaEvent_t a = nullptr, b = nullptr;
    if ((e = cudaEventCreate(&a)) || (e = cudaEventCreate(&b))) return fail(e);
    // best of two timed forwards (after one warm-up) over the first nt trials
    auto time_shape = [&](const std::array<int32_t, 5>& c, int64_t nt, float& ms_best) -> cudaError_t {
        YetArgs yt = y;
        yt.n_trials = nt;
        cudaError_t err = apply_shape(p, c.data());
        if (!err) err = run_forward(p, c[0], yt, ylt_dev, nullptr, stream);  // warm-up
        ms_best = -1.0f;
        for (int r = 0; r < 2 && !err; ++r) {
            cudaEventRecord(a, stream);
            err = run_forward(p, c[0], yt, ylt_dev, nullptr, stream);
            cudaEventRecord(b, stream);
            if (!err) err = cudaEventSynchronize(b);
            float ms = 0.0f;
            if (!err) cudaEventElapsedTime(&ms, a, b);
            if (ms_best < 0 || ms < ms_best) ms_best = ms;
        }
        return err;
    };
    std::vector<float> sample(cands.size(), -1.0f);
    for (size_t ci = 0; ci < cands.size() && !e; ++ci) {
        if ((e = time_shape(cands[ci], ts, sample[ci]))) break;
        ++res.candidates;
    }
    // A call has a part that does not grow with the trials (the skip
    // variant's occurrence-table build, launch and fill costs). Per variant,
    // its fastest shape is timed again on twice the sample, which separates
    // that part (2 t(s) - t(2s)) from the per-trial part; every candidate is
    // then ranked by its time extrapolated to n_trials.
    float fixed[6] = {0, 0, 0, 0, 0, 0};
    if (!e && n_trials >= 2 * ts) {
        for (int v = ART_VARIANT_PLAIN; v <= ART_VARIANT_SPARSE && !e; ++v) {
            int bi = -1;
            for (size_t ci = 0; ci < cands.size(); ++ci)
                if (cands[ci][0] == v && (bi < 0 || sample[ci] < sample[bi])) bi = (int)ci;
            if (bi < 0) continue;
            float t2 = 0.0f;
            if ((e = time_shape(cands[bi], 2 * ts, t2))) break;
            fixed[v] = std::max(0.0f, std::min(sample[bi], 2.0f * sample[bi] - t2));
        }
    }
    float best_ms = -1.0f, best_pred = -1.0f;
    for (size_t ci = 0; ci < cands.size() && !e; ++ci) {
        const float f = fixed[cands[ci][0]];
        const float pred = f + (sample[ci] - f) * (float)((double)n_trials / (double)ts);
        if (best_pred < 0 || pred < best_pred) {
            best_pred = pred;
            best_ms = sample[ci];
            std::copy(cands[ci].begin(), cands[ci].end(), best);
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e) {
        apply_shape(p, saved);
        return fail(e);
    }
    if (best_ms < 0) return ART_EUNSUPPORTED;
    if ((e = apply_shape(p, best))) return fail(e);
    cache_store(key, best, best_ms);
    res.variant = best[0]; res.slots = best[1]; res.trial_tile = best[2]; res.cta_threads = best[3];
    res.mapping = best[4];
    res.sample_ms = best_ms;
    if (out) *out = res;
    return ART_OK;
}

}  // extern "C"

// probes.cu -- measurements of the limits the ARA kernels run against (the
// paper has no counterpart; they give the roofline denominators that a
// device's copy-bandwidth and GEMM peaks do not cover).
//
//   ART_PROBE_STREAM     streaming read of a buffer (GB/s of buffer bytes)
//   ART_PROBE_GATHER32   random 32-byte sector reads over a buffer (GB/s of
//                        sector bytes); a buffer below the L2 size measures
//                        the L2 gather rate, one far above it the DRAM rate
//   ART_PROBE_GATHER64   the same with 64-byte rows (two sectors per read)
//   ART_PROBE_GATHER4    random 4-byte reads (GB/s of 32-byte sectors touched)
//   ART_PROBE_FP64ADD    dependent-free FP64 adds (GFLOP/s)
// Each probe runs `reps` timed launches after one warm-up and returns the
// best. Positions come from a counter hash (splitmix64 finaliser), so every
// launch reads the same addresses.
#include <algorithm>

#include "art_internal.cuh"

namespace art {
namespace {

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void fill_kernel(float* p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (float)(i & 1023) * 0.5f;
}

__global__ void stream_kernel(const float4* __restrict__ p, int64_t n4, float* __restrict__ sink) {
    float acc = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = __ldcs(p + i);
        acc += v.x + v.y + v.z + v.w;
    }
    if (acc == -1.0f) *sink = acc;  // keeps the loads; never true for this data
}

// Each thread issues `per` independent reads of `width` floats at hashed,
// width-aligned positions of a buffer of n floats.
template <int WIDTH>
__global__ void gather_kernel(const float* __restrict__ p, int64_t n, int per, float* __restrict__ sink) {
    const int64_t slots = n / WIDTH;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.0f;
    for (int r = 0; r < per; r += 4) {
        float v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t slot = (int64_t)(mix64(tid * 1315423911ull + r + u) % (uint64_t)slots);
            const float* q = p + slot * WIDTH;
            if constexpr (WIDTH == 16) {
                float w[8], z[8];
                asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                    : "=f"(w[0]), "=f"(w[1]), "=f"(w[2]), "=f"(w[3]), "=f"(w[4]), "=f"(w[5]), "=f"(w[6]), "=f"(w[7])
                    : "l"(q));
                asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                    : "=f"(z[0]), "=f"(z[1]), "=f"(z[2]), "=f"(z[3]), "=f"(z[4]), "=f"(z[5]), "=f"(z[6]), "=f"(z[7])
                    : "l"(q + 8));
                v[u] = w[0] + w[7] + z[0] + z[7];
            } else if constexpr (WIDTH == 8) {
                float w[8];
                asm("ld.global.nc.L1::no_allocate.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                    : "=f"(w[0]), "=f"(w[1]), "=f"(w[2]), "=f"(w[3]), "=f"(w[4]), "=f"(w[5]), "=f"(w[6]), "=f"(w[7])
                    : "l"(q));
                v[u] = w[0] + w[7];
            } else {
                v[u] = __ldg(q);
            }
        }
        acc += v[0] + v[1] + v[2] + v[3];
    }
    if (acc == -1.0f) *sink = acc;
}

__global__ void fp64_kernel(int iters, double* sink) {
    double a0 = threadIdx.x * 1e-9, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6,
           a7 = a0 + 7;
    const double d = 1e-12;
    for (int i = 0; i < iters; ++i) {
        a0 += d; a1 += d; a2 += d; a3 += d; a4 += d; a5 += d; a6 += d; a7 += d;
    }
    const double s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
    if (s == -1.0) *sink = s;
}

}  // namespace
}  // namespace art

using namespace art;

extern "C" art_status art_probe(int32_t kind, int64_t bytes, int32_t reps, double* result) {
    if (!result || reps < 1 || kind < ART_PROBE_STREAM || kind > ART_PROBE_FP64ADD) return ART_EINVAL;
    if (kind != ART_PROBE_FP64ADD && (bytes < (1 << 20) || bytes > ((int64_t)64 << 30))) return ART_EINVAL;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (!e) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e) {
        set_last_error(e);
        return ART_ECUDA;
    }
    float* buf = nullptr;
    float* sink = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    const int64_t n = bytes / 4;
    if ((e = cudaMalloc(&sink, 64))) goto done;
    if (kind != ART_PROBE_FP64ADD) {
        if ((e = cudaMalloc(&buf, (size_t)n * 4))) goto done;
        fill_kernel<<<sms * 8, 256>>>(buf, n);
    }
    if ((e = cudaEventCreate(&a)) || (e = cudaEventCreate(&b))) goto done;
    {
        double best = 0.0;
        const int per = 64;
        const int64_t threads = (int64_t)sms * 2048;
        for (int r = 0; r <= reps; ++r) {
            cudaEventRecord(a);
            double amount = 0.0;
            switch (kind) {
                case ART_PROBE_STREAM:
                    stream_kernel<<<sms * 8, 256>>>(reinterpret_cast<const float4*>(buf), n / 4, sink);
                    amount = (double)(n / 4) * 16.0;
                    break;
                case ART_PROBE_GATHER32:
                    gather_kernel<8><<<(unsigned)(threads / 256), 256>>>(buf, n, per, sink);
                    amount = (double)threads * per * 32.0;
                    break;
                case ART_PROBE_GATHER64:
                    gather_kernel<16><<<(unsigned)(threads / 256), 256>>>(buf, n, per, sink);
                    amount = (double)threads * per * 64.0;
                    break;
                case ART_PROBE_GATHER4:
                    gather_kernel<1><<<(unsigned)(threads / 256), 256>>>(buf, n, per, sink);
                    amount = (double)threads * per * 32.0;
                    break;
                case ART_PROBE_FP64ADD: {
                    const int iters = 4096;
                    fp64_kernel<<<sms * 16, 256>>>(iters, reinterpret_cast<double*>(sink));
                    amount = (double)sms * 16 * 256 * iters * 8.0;
                    break;
                }
            }
            cudaEventRecord(b);
            if ((e = cudaEventSynchronize(b))) goto done;
            if ((e = cudaGetLastError())) goto done;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, a, b);
            if (r > 0 && ms > 0.0f) best = std::max(best, amount / (ms * 1e-3) / 1e9);
        }
        *result = best;
    }
done:
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaFree(buf);
    cudaFree(sink);
    if (e) {
        set_last_error(e);
        return e == cudaErrorMemoryAllocation ? ART_ENOMEM : ART_ECUDA;
    }
    return ART_OK;
}

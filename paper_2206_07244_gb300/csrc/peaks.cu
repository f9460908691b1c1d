// Throughput probes of the operations the numeric kernels are built from:
// float64 fused multiply-add, float64 accumulation in shared memory (the
// compare-and-swap loop the kernels use, and the native atomic add), 32-bit
// shared atomics, and float64 reductions in global memory (L2). Each probe
// keeps every SM busy with one 1024-thread block and reports operations per
// second. `hot` sets the contention: 0 spreads the addresses uniformly over
// the probe's array, h > 0 sends every operation to one of h addresses.
//
// These give the ceilings that the numeric phase's roofline is read against:
// every intermediate product costs one float64 multiply-add and one
// accumulation into its output entry, whatever the memory system does.
#include <algorithm>
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "opsparse.h"

namespace ops {
namespace {

constexpr int kProbeBlock = 1024;
constexpr int kProbeSmemDoubles = 16384;   // 128 KB

__device__ __forceinline__ uint32_t lcg(uint32_t &x) {
    x = x * 1664525u + 1013904223u;
    return x;
}

// index in [0, n) (n a power of two) or one of `hot` addresses spread over n
__device__ __forceinline__ uint32_t pick(uint32_t &x, int lgn, int hot) {
    const uint32_t r = lcg(x);
    if (hot <= 0) return r >> (32 - lgn);
    const uint32_t k = (r >> 8) % static_cast<uint32_t>(hot);
    return (k * 2654435761u) >> (32 - lgn);
}

__global__ void __launch_bounds__(kProbeBlock, 1) probe_fma(long long iters, double *sink) {
    double a[8];
    const double b = 1.0000001 + threadIdx.x * 1e-12, c = 1e-9;
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = j + threadIdx.x * 1e-6;
    for (long long i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += a[j];
    if (sink && s == 12345.678) sink[0] = s;   // keeps the chains alive
}

template <int OP>
__global__ void __launch_bounds__(kProbeBlock, 1) probe_smem(long long iters, int hot, double *sink) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *t = reinterpret_cast<double *>(smem_raw);
    unsigned *u = reinterpret_cast<unsigned *>(smem_raw);
    int *k = reinterpret_cast<int *>(smem_raw);
    for (int i = threadIdx.x; i < kProbeSmemDoubles; i += kProbeBlock) t[i] = 0.0;
    __syncthreads();
    uint32_t x = 0x9E3779B9u * (blockIdx.x * kProbeBlock + threadIdx.x + 1);
    const double a = 0.5 + threadIdx.x * 1e-9, b = 0.25;
    int found = 0;
    for (long long i = 0; i < iters; ++i) {
        if (OP == 1) {
            smem_fma_add(t + pick(x, 14, hot), a, b);
        } else if (OP == 2) {
            atomicAdd(t + pick(x, 14, hot), a * b);
        } else if (OP == 3) {
            const uint32_t j = pick(x, 19, hot);   // 2^19 bits over the 64 KB of words
            atomicOr(u + (j >> 5), 1u << (j & 31));
        } else {
            const uint32_t j = pick(x, 15, hot);   // 2^15 int slots
            found += atomicCAS(k + j, 0, 1);
        }
    }
    __syncthreads();
    if (sink && threadIdx.x == 0 && (t[0] == 12345.678 || found == -7)) sink[0] = t[1];
}

// COAL: the 32 lanes of a warp reduce into 32 consecutive doubles (one
// random base per warp and step) instead of 32 independent addresses.
template <int UNROLL, bool COAL>
__global__ void __launch_bounds__(kProbeBlock, 1) probe_red(long long iters, int hot, double *buf, int lgn) {
    const int lane = threadIdx.x & 31;
    uint32_t x = 0x9E3779B9u * (blockIdx.x * kProbeBlock + (COAL ? threadIdx.x >> 5 : threadIdx.x) + 1);
    const double v = 1e-9 * (threadIdx.x + 1);
    for (long long i = 0; i < iters; i += UNROLL) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            uint32_t j = pick(x, lgn, hot);
            if (COAL) j = (j & ~31u) + lane;
            asm volatile("red.global.add.f64 [%0], %1;" ::"l"(buf + j), "d"(v) : "memory");
        }
    }
}

}  // namespace
}  // namespace ops

using namespace ops;

extern "C" int spgemm_probe(int op, int hot, int64_t iters, void *buf, int64_t buf_bytes, double *gops,
                            void *stream) {
    if (!gops || iters <= 0 || hot < 0 || op < 0 || op > 7) return SPGEMM_ERR_INVALID;
    if (op >= 5 && (!buf || buf_bytes < (1 << 20))) return SPGEMM_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SPGEMM_ERR_CUDA;
    double *sink = static_cast<double *>(buf);
    const size_t smem = sizeof(double) * kProbeSmemDoubles;
    // largest power of two of doubles that fits the buffer (L2-resident size for op 5)
    int lgn = 0;
    if (buf) {
        const int64_t cap = op == 5 || op == 7 ? std::min<int64_t>(buf_bytes, 32ll << 20) : buf_bytes;
        while ((int64_t{8} << (lgn + 1)) <= cap && lgn < 31) ++lgn;
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SPGEMM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return SPGEMM_ERR_CUDA;
    }
    cudaError_t err = cudaSuccess;
    auto launch = [&]() {
        switch (op) {
            case 0: probe_fma<<<sms, kProbeBlock, 0, s>>>(iters, sink); break;
            case 1: probe_smem<1><<<sms, kProbeBlock, smem, s>>>(iters, hot, sink); break;
            case 2: probe_smem<2><<<sms, kProbeBlock, smem, s>>>(iters, hot, sink); break;
            case 3: probe_smem<3><<<sms, kProbeBlock, smem, s>>>(iters, hot, sink); break;
            case 4: probe_smem<4><<<sms, kProbeBlock, smem, s>>>(iters, hot, sink); break;
            case 7: probe_red<4, true><<<sms, kProbeBlock, 0, s>>>(iters, hot, static_cast<double *>(buf), lgn); break;
            default: probe_red<4, false><<<sms, kProbeBlock, 0, s>>>(iters, hot, static_cast<double *>(buf), lgn); break;
        }
        return cudaGetLastError();
    };
    for (int k = 1; k <= 4 && err == cudaSuccess; ++k)
        err = cudaFuncSetAttribute(reinterpret_cast<const void *>(
                                       k == 1 ? probe_smem<1> : k == 2 ? probe_smem<2> : k == 3 ? probe_smem<3>
                                                                                                   : probe_smem<4>),
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err == cudaSuccess && op >= 5) err = cudaMemsetAsync(buf, 0, static_cast<size_t>(buf_bytes), s);
    if (err == cudaSuccess) err = launch();   // warm-up
    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
    if (err == cudaSuccess) err = launch();
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return SPGEMM_ERR_CUDA;
    const double ops_total = static_cast<double>(sms) * kProbeBlock * static_cast<double>(iters) * (op == 0 ? 8.0 : 1.0);
    *gops = ops_total / (ms * 1e-3) / 1e9;
    return SPGEMM_OK;
}

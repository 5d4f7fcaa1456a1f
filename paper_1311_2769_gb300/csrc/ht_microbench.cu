// ht_microbench.cu — throughput ceilings of the operations the vote is made
// of, measured on the GPU the library runs on: FP32 multiply/add lane
// operations, predicated shared-memory reductions (the vote's increment) at
// random addresses of an accumulator tile, IEEE float32 divisions, and
// binary64 multiply/add (the circle fit's and the merge's arithmetic).  The
// kernels' fractions of these ceilings say which one binds them.
#include <cuda_runtime.h>

#include <cstdint>

#include "ht_internal.h"

namespace ht {
namespace {

constexpr int kMbBlocksPerSm = 8;
constexpr int kMbThreads = 256;
constexpr int kMbTableWords = 4096;  // 16 KB accumulator tile per block

// 8 independent chains of one multiply and one add each (no contraction).
__global__ void mb_fp32_kernel(int64_t iters, float seed, float* sink) {
    float a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = seed + (float)(threadIdx.x + c);
    const float m = 0.999f, k = 1e-3f;
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = __fadd_rn(__fmul_rn(a[c], m), k);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    if (s == 12345.678f) sink[blockIdx.x] = s;  // keeps the chains live
}

// 8 independent chains of one binary64 multiply and one add each.
__global__ void mb_fp64_kernel(int64_t iters, float seed, float* sink) {
    double a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = (double)seed + (double)(threadIdx.x + c);
    const double m = 0.999, k = 1e-3;
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = __dadd_rn(__dmul_rn(a[c], m), k);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    if (s == 12345.678) sink[blockIdx.x] = (float)s;
}

// 8 independent chains of IEEE divisions x -> k / x (stays finite).
__global__ void mb_fdiv_kernel(int64_t iters, float seed, float* sink) {
    float a[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) a[c] = seed + (float)(threadIdx.x + c);
    const float k = 3.0f;
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < 8; ++c) a[c] = __fdiv_rn(k, a[c]);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += a[c];
    if (s == 12345.678f) sink[blockIdx.x] = s;
}

// red.shared.add.u32 at pseudo-random addresses of a 4096-word tile, 8 per
// iteration per thread; the tile's total is written out so nothing is dead.
__global__ void mb_red_kernel(int64_t iters, float seed, float* sink) {
    __shared__ uint32_t table[kMbTableWords];
    for (int i = threadIdx.x; i < kMbTableWords; i += blockDim.x) table[i] = 0;
    __syncthreads();
    uint32_t x = 2463534242u ^ (blockIdx.x * 7919u + threadIdx.x * 104729u) ^ (uint32_t)seed;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(table);
    for (int64_t t = 0; t < iters; ++t) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            x ^= x << 13;
            x ^= x >> 17;
            x ^= x << 5;
            const uint32_t addr = base + 4u * (x & (kMbTableWords - 1));
            asm volatile("red.shared.add.u32 [%0], 1;" ::"r"(addr) : "memory");
        }
    }
    __syncthreads();
    uint32_t s = 0;
    for (int i = threadIdx.x; i < kMbTableWords; i += blockDim.x) s += table[i];
    if (s == 0xFFFFFFFFu) sink[blockIdx.x] = (float)s;
}

}  // namespace

cudaError_t run_microbench(int kind, int64_t iters, int sms, float* sink, float* ms, double* ops) {
    const int blocks = sms * kMbBlocksPerSm;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e) return e;
    e = cudaEventCreate(&e1);
    if (e) {
        cudaEventDestroy(e0);
        return e;
    }
    auto launch = [&](int64_t n) {
        if (kind == 0) mb_fp32_kernel<<<blocks, kMbThreads>>>(n, 1.0f, sink);
        else if (kind == 1) mb_red_kernel<<<blocks, kMbThreads>>>(n, 1.0f, sink);
        else if (kind == 2) mb_fdiv_kernel<<<blocks, kMbThreads>>>(n, 1.0f, sink);
        else mb_fp64_kernel<<<blocks, kMbThreads>>>(n, 1.0f, sink);
    };
    launch(iters / 8 + 1);  // warm-up
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    e = cudaGetLastError();
    if (!e) e = cudaEventSynchronize(e1);
    if (!e) e = cudaEventElapsedTime(ms, e0, e1);
    const double per_iter = (kind == 0 || kind == 3) ? 16.0 : 8.0;  // 8 chains x (mul + add)
    *ops = (double)blocks * kMbThreads * (double)iters * per_iter;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e;
}

}  // namespace ht

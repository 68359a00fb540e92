// Integer-throughput probes for the integer-pipe roofline of the sweep: the
// sweep's word logic is 3-input logic (ALU pipe), its site mapping and Philox
// multiplies are integer multiply-adds (FMA pipe), and Philox-4x32-10 is most
// of its integer work.  Each probe runs a fixed chain of instructions that no
// compiler pass can shorten (every result feeds later instructions, every
// instruction has three distinct live inputs) on every SM, and the host times
// it with CUDA events.
#include <cuda_runtime.h>

#include "../../include/rsos.h"
#include "philox.cuh"

namespace {

constexpr int kChains = 8;

// kind 0: lop3 (xor of three), kind 1: mad.lo (a * b + c); 8 per iteration.
template <int KIND>
__global__ void __launch_bounds__(256) peak_int_kernel(uint32_t seed, int iters, uint32_t* sink)
{
    uint32_t r[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) r[k] = seed ^ (threadIdx.x * 0x9E3779B9u) ^ (blockIdx.x * 0x85EBCA6Bu) ^ (k * 0x27D4EB2Fu) | 1u;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            if (KIND == 0)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(r[k]) : "r"(r[(k + 1) % kChains]), "r"(r[(k + 3) % kChains]));
            else
                asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(r[k]) : "r"(r[(k + 1) % kChains]), "r"(r[(k + 3) % kChains]));
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc ^= r[k];
    if (acc == seed) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;  // keeps the chains live
}

// Philox-4x32-10 blocks with precomputed round keys, as the sweep draws them.
__global__ void __launch_bounds__(256) peak_philox_kernel(uint32_t seed, int iters, uint32_t* sink)
{
    const rsos::RoundKeys rk = rsos::philox_round_keys(seed, seed ^ 0x5bd1e995u);
    const uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t acc = 0;
    for (int i = 0; i < iters; ++i) {
        const rsos::U4 v = rsos::philox4x32_10(rsos::U4{id, (uint32_t)i, seed, 2u << 30}, rk);
        acc ^= v.x ^ v.y ^ v.z ^ v.w;
    }
    if (acc == seed) sink[id] = acc;
}

}  // namespace

extern "C" int rsos_peak_int(int32_t kind, int64_t iters, double* per_s, void* stream)
{
    if (kind < 0 || kind > 2 || iters < 1 || iters > (1 << 30) || !per_s) return RSOS_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        (void)cudaGetLastError();
        return RSOS_ECUDA;
    }
    const int threads = 256, blocks = sms * 8;  // 2048 threads per SM, full occupancy
    uint32_t* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&sink, (size_t)blocks * threads * 4);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    auto launch = [&](int n) {
        if (kind == 0) peak_int_kernel<0><<<blocks, threads, 0, s>>>(0x2016u, n, sink);
        else if (kind == 1) peak_int_kernel<1><<<blocks, threads, 0, s>>>(0x2016u, n, sink);
        else peak_philox_kernel<<<blocks, threads, 0, s>>>(0x2016u, n, sink);
        return cudaGetLastError();
    };
    if (e == cudaSuccess) e = launch(iters > 16 ? 16 : (int)iters);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch((int)iters);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (e != cudaSuccess || ms <= 0.f) {
        (void)cudaGetLastError();
        return RSOS_ECUDA;
    }
    const double units = (double)blocks * threads * (double)iters * (kind == 2 ? 1.0 : (double)kChains);
    *per_s = units / (ms * 1e-3);
    return RSOS_OK;
}

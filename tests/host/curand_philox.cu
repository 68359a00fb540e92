// Test helper: cuRAND's device Philox-4x32-10 block function evaluated on
// caller-given (counter, key) pairs, so the oracle's generator can be
// compared with an independent implementation.  Not part of the library.
#include <cstdint>
#include <cuda_runtime.h>
#include <curand_kernel.h>

__global__ void blocks(const uint4* ctr, const uint2* key, uint4* out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(ctr[i], key[i]);
}

extern "C" int curand_philox_blocks(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n)
{
    uint4 *dc = nullptr, *dout = nullptr;
    uint2* dk = nullptr;
    cudaError_t e = cudaMalloc(&dc, (size_t)n * 16);
    if (e == cudaSuccess) e = cudaMalloc(&dk, (size_t)n * 8);
    if (e == cudaSuccess) e = cudaMalloc(&dout, (size_t)n * 16);
    if (e == cudaSuccess) e = cudaMemcpy(dc, ctr, (size_t)n * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dk, key, (size_t)n * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        blocks<<<(n + 255) / 256, 256>>>(dc, dk, dout, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, (size_t)n * 16, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dk);
    cudaFree(dout);
    return (int)e;
}

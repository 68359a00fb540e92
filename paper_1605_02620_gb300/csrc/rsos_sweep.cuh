// Phase kernels of the double-tiling sweep: one launch activates the
// sub-tile set q = perm[p] of every tile (section II), one thread per
// (tile, lane-word group).  Included by one translation unit per SX.
#pragma once
#include "rsos_launch.h"

namespace rsos {

template <int N, typename WT, int SX>
__global__ void __launch_bounds__(512) phase_kernel(JobDev J, uint32_t t, int p, int q, int ox, int oy,
                                                     Origin00 o)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WT* sm = reinterpret_cast<WT*>(smem_raw);
    const int nthr = blockDim.x, tid = threadIdx.x;
    const long long gid = (long long)blockIdx.x * nthr + tid;
    const long long per_row = (long long)J.nT * J.NWP;
    if (gid >= per_row * J.nT) return;
    const int ty = (int)(gid / per_row);
    const int rem = (int)(gid - (long long)ty * per_row);
    const int tx = rem / J.NWP, wp = rem - tx * J.NWP;
    if (q == o.q && tx == o.tx && ty == o.ty) {
        activate_subtile<N, WT, SX, true>(J, sm, tid, nthr, tx, ty, wp, t, p, q, ox, oy, o.k);
    } else {
        activate_subtile<N, WT, SX, false>(J, sm, tid, nthr, tx, ty, wp, t, p, q, ox, oy, -1);
    }
}

template <int SX>
__global__ void __launch_bounds__(512) plain_phase_kernel(JobDev J, uint32_t t, int p, int q, int ox, int oy)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int32_t* sm = reinterpret_cast<int32_t*>(smem_raw);
    const int nthr = blockDim.x, tid = threadIdx.x;
    const long long gid = (long long)blockIdx.x * nthr + tid;
    if (gid >= (long long)J.nT * J.nT) return;
    const int ty = (int)(gid / J.nT), tx = (int)(gid - (long long)ty * J.nT);
    activate_subtile_plain<SX>(J, sm, tid, nthr, tx, ty, t, p, q, ox, oy);
}

// Largest dynamic shared memory of one block (227 KB).
constexpr size_t kMaxDynamicSmem = 227 * 1024;

inline int pick_threads(size_t per_thread, size_t smem_budget, long long total)
{
    long long n = (long long)(smem_budget / per_thread) / 32 * 32;
    if (n > 512) n = 512;
    if (n < 32) n = 32;
    const long long need = (total + 31) / 32 * 32;
    if (need < n) n = need < 32 ? 32 : need;
    return (int)n;
}

template <int N, typename WT, int SX>
cudaError_t launch_phase_t(const JobDev& J, uint32_t t, int p, int q, int ox, int oy, const Origin00& o,
                           size_t smem_budget, cudaStream_t s)
{
    constexpr int B = bits_for_step(N);
    const size_t per_thread = (size_t)(SX + 2) * (SX + 2) * B * sizeof(WT);
    const long long total = (long long)J.nT * J.nT * J.NWP;
    const int nthr = pick_threads(per_thread, smem_budget, total);
    const size_t smem = per_thread * nthr;
    // Allow the largest dynamic shared memory once (thread-safe static
    // initialisation; handles on different host threads launch concurrently).
    static const cudaError_t allowed = cudaFuncSetAttribute(
        phase_kernel<N, WT, SX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDynamicSmem);
    if (allowed != cudaSuccess) return allowed;
    const long long blocks = (total + nthr - 1) / nthr;
    phase_kernel<N, WT, SX><<<(unsigned)blocks, nthr, smem, s>>>(J, t, p, q, ox, oy, o);
    return cudaGetLastError();
}

template <int SX>
cudaError_t launch_phase_sx(const JobDev& J, int words_per_thread, uint32_t t, int p, int q, int ox, int oy,
                            const Origin00& o, size_t smem_budget, cudaStream_t s)
{
#define RSOS_CASE(NN)                                                                                  \
    case NN:                                                                                           \
        return words_per_thread == 2                                                                   \
                   ? launch_phase_t<NN, uint64_t, SX>(J, t, p, q, ox, oy, o, smem_budget, s)           \
                   : launch_phase_t<NN, uint32_t, SX>(J, t, p, q, ox, oy, o, smem_budget, s);
    switch (J.N) {
        RSOS_CASE(1)
        RSOS_CASE(2)
        RSOS_CASE(3)
        RSOS_CASE(4)
        RSOS_CASE(5)
        RSOS_CASE(6)
        RSOS_CASE(7)
        default:
            return cudaErrorInvalidValue;
    }
#undef RSOS_CASE
}

template <int SX>
cudaError_t launch_plain_sx(const JobDev& J, uint32_t t, int p, int q, int ox, int oy, size_t smem_budget,
                            cudaStream_t s)
{
    const size_t per_thread = (size_t)(SX + 2) * (SX + 2) * sizeof(int32_t);
    const long long total = (long long)J.nT * J.nT;
    const int nthr = pick_threads(per_thread, smem_budget, total);
    const size_t smem = per_thread * nthr;
    static const cudaError_t allowed = cudaFuncSetAttribute(
        plain_phase_kernel<SX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxDynamicSmem);
    if (allowed != cudaSuccess) return allowed;
    const long long blocks = (total + nthr - 1) / nthr;
    plain_phase_kernel<SX><<<(unsigned)blocks, nthr, smem, s>>>(J, t, p, q, ox, oy);
    return cudaGetLastError();
}

}  // namespace rsos

#define RSOS_DEFINE_SX(SX)                                                                            \
    namespace rsos {                                                                                  \
    cudaError_t launch_phase_s##SX(const JobDev& J, int words_per_thread, uint32_t t, int p, int q,   \
                                   int ox, int oy, const Origin00& o, size_t smem_budget,            \
                                   cudaStream_t s)                                                    \
    {                                                                                                 \
        return launch_phase_sx<SX>(J, words_per_thread, t, p, q, ox, oy, o, smem_budget, s);          \
    }                                                                                                 \
    cudaError_t launch_phase_plain_s##SX(const JobDev& J, uint32_t t, int p, int q, int ox, int oy,   \
                                         size_t smem_budget, cudaStream_t s)                          \
    {                                                                                                 \
        return launch_plain_sx<SX>(J, t, p, q, ox, oy, smem_budget, s);                               \
    }                                                                                                 \
    }

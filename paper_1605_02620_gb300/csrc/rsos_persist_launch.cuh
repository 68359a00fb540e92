// Host launchers of the persistent engine, instantiated per sub-tile edge SX
// in rsos_persist_s{1,2,4,8}.cu.
#pragma once
#include <cstdlib>

#include "rsos_launch.h"

namespace rsos {

template <int N, typename WT, int SX>
cudaError_t plan_persist_t(const JobDev& J, int block_tiles, int phase_lag, PersistPlan* P)
{
    constexpr int B = bits_for_step(N);
    constexpr int WPB = PersistCfg<N, WT, SX>::WPB;
    const size_t per_thread = (size_t)PersistCfg<N, WT, SX>::SLOTS * B * sizeof(WT);
    P->CW = block_tiles;  // TPL * (32 / NWP), fixed by the job layout
    if (P->CW < 1) return cudaErrorInvalidConfiguration;
    P->K = (J.nT + P->CW - 1) / P->CW;
    P->nthr = 32 * WPB;
    P->smem = per_thread * (size_t)P->nthr;
    cudaError_t e = cudaFuncSetAttribute(persistent_kernel<N, WT, SX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)P->smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_kernel<N, WT, SX>, P->nthr, P->smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int dev = 0, sms = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    P->grid = per_sm * sms;
    // Phase lag D (slots between consecutive phase fronts).  A dependency sits
    // about D slots (D * 4K tickets) behind its dependant; with two tickets
    // per worker warp in flight, D = 1.5 * in-flight / (4K) keeps dependencies
    // complete by the time they are checked (L = 4096, N = 1, 64 surfaces:
    // D = nT / 3 = 170; measured flat from 150 to 340, 6% slower at 91, 24%
    // at 48).  The rows between the fronts need not fit in L2: with 16-byte
    // site records the re-reads cost less than the waits a short lag causes.
    const int per_slot = 4 * P->K;
    const int workers = P->grid * WPB;
    int D = (int)(1.5 * 2.0 * workers / per_slot);
    const int dmax = J.nT / 3 > 2 ? J.nT / 3 : 2;
    if (D > dmax) D = dmax;
    if (D < 2) D = 2;
    if (const char* env = getenv("RSOS_PHASE_LAG")) {
        const int v = atoi(env);
        if (v >= 2) D = v;
    }
    if (phase_lag >= 2) D = phase_lag;
    P->D = D;
    return cudaSuccess;
}

template <int N, typename WT, int SX>
cudaError_t launch_persist_t(const PersistArgs& A, const PersistPlan& P, cudaStream_t s)
{
    PersistArgs a = A;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)persistent_kernel<N, WT, SX>, dim3(P.grid), dim3(P.nthr), args,
                                       P.smem, s);
}

template <int N, typename WT, int SX>
cudaError_t plan_multi_t(int* grid, int* block, size_t* smem)
{
    constexpr int B = bits_for_step(N);
    constexpr int WPB = PersistCfg<N, WT, SX>::WPB;
    *block = 32 * WPB;
    *smem = (size_t)PersistCfg<N, WT, SX>::SLOTS * B * sizeof(WT) * (size_t)(*block);
    cudaError_t e = cudaFuncSetAttribute(persistent_multi_kernel<N, WT, SX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)*smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_multi_kernel<N, WT, SX>, *block, *smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *grid = per_sm * sms;
    return cudaSuccess;
}

template <int N, typename WT, int SX>
cudaError_t launch_multi_t(const MultiArgs& M, int grid, int block, size_t smem, cudaStream_t s)
{
    MultiArgs a = M;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)persistent_multi_kernel<N, WT, SX>, dim3(grid), dim3(block), args,
                                       smem, s);
}

#define RSOS_PERSIST_SWITCH(CALL_U64, CALL_U32)                                                       \
    switch (J.N) {                                                                                     \
        case 1: return words_per_thread == 2 ? CALL_U64(1) : CALL_U32(1);                              \
        case 2: return words_per_thread == 2 ? CALL_U64(2) : CALL_U32(2);                              \
        case 3: return words_per_thread == 2 ? CALL_U64(3) : CALL_U32(3);                              \
        case 4: return words_per_thread == 2 ? CALL_U64(4) : CALL_U32(4);                              \
        case 5: return words_per_thread == 2 ? CALL_U64(5) : CALL_U32(5);                              \
        case 6: return words_per_thread == 2 ? CALL_U64(6) : CALL_U32(6);                              \
        case 7: return words_per_thread == 2 ? CALL_U64(7) : CALL_U32(7);                              \
        default: return cudaErrorInvalidValue;                                                         \
    }

template <int SX>
cudaError_t plan_persist_sx(const JobDev& J, int words_per_thread, int block_tiles, int phase_lag, PersistPlan* out)
{
#define RSOS_P64(NN) plan_persist_t<NN, uint64_t, SX>(J, block_tiles, phase_lag, out)
#define RSOS_P32(NN) plan_persist_t<NN, uint32_t, SX>(J, block_tiles, phase_lag, out)
    RSOS_PERSIST_SWITCH(RSOS_P64, RSOS_P32)
#undef RSOS_P64
#undef RSOS_P32
}

template <int SX>
cudaError_t launch_persist_sx(const JobDev& J, int words_per_thread, const PersistArgs& A, const PersistPlan& P,
                              cudaStream_t s)
{
#define RSOS_L64(NN) launch_persist_t<NN, uint64_t, SX>(A, P, s)
#define RSOS_L32(NN) launch_persist_t<NN, uint32_t, SX>(A, P, s)
    RSOS_PERSIST_SWITCH(RSOS_L64, RSOS_L32)
#undef RSOS_L64
#undef RSOS_L32
}

#define RSOS_MULTI_SWITCH(CALL_U64, CALL_U32)                                                         \
    switch (N) {                                                                                       \
        case 1: return words_per_thread == 2 ? CALL_U64(1) : CALL_U32(1);                              \
        case 2: return words_per_thread == 2 ? CALL_U64(2) : CALL_U32(2);                              \
        case 3: return words_per_thread == 2 ? CALL_U64(3) : CALL_U32(3);                              \
        case 4: return words_per_thread == 2 ? CALL_U64(4) : CALL_U32(4);                              \
        case 5: return words_per_thread == 2 ? CALL_U64(5) : CALL_U32(5);                              \
        case 6: return words_per_thread == 2 ? CALL_U64(6) : CALL_U32(6);                              \
        case 7: return words_per_thread == 2 ? CALL_U64(7) : CALL_U32(7);                              \
        default: return cudaErrorInvalidValue;                                                         \
    }

template <int SX>
cudaError_t plan_multi_sx(int N, int words_per_thread, int* grid, int* block, size_t* smem)
{
#define RSOS_M64(NN) plan_multi_t<NN, uint64_t, SX>(grid, block, smem)
#define RSOS_M32(NN) plan_multi_t<NN, uint32_t, SX>(grid, block, smem)
    RSOS_MULTI_SWITCH(RSOS_M64, RSOS_M32)
#undef RSOS_M64
#undef RSOS_M32
}

template <int SX>
cudaError_t launch_multi_sx(int N, int words_per_thread, const MultiArgs& M, int grid, int block, size_t smem,
                            cudaStream_t s)
{
#define RSOS_L64(NN) launch_multi_t<NN, uint64_t, SX>(M, grid, block, smem, s)
#define RSOS_L32(NN) launch_multi_t<NN, uint32_t, SX>(M, grid, block, smem, s)
    RSOS_MULTI_SWITCH(RSOS_L64, RSOS_L32)
#undef RSOS_L64
#undef RSOS_L32
}

}  // namespace rsos

#define RSOS_DEFINE_PERSIST(SX)                                                                       \
    namespace rsos {                                                                                  \
    cudaError_t plan_persist_s##SX(const JobDev& J, int words_per_thread, int block_tiles, int phase_lag, \
                                   PersistPlan* out)                                                  \
    {                                                                                                 \
        return plan_persist_sx<SX>(J, words_per_thread, block_tiles, phase_lag, out);                 \
    }                                                                                                 \
    cudaError_t launch_persist_s##SX(const JobDev& J, int words_per_thread, const PersistArgs& A,     \
                                     const PersistPlan& P, cudaStream_t s)                            \
    {                                                                                                 \
        return launch_persist_sx<SX>(J, words_per_thread, A, P, s);                                   \
    }                                                                                                 \
    cudaError_t plan_multi_s##SX(int N, int words_per_thread, int* grid, int* block, size_t* smem)    \
    {                                                                                                 \
        return plan_multi_sx<SX>(N, words_per_thread, grid, block, smem);                             \
    }                                                                                                 \
    cudaError_t launch_multi_s##SX(int N, int words_per_thread, const MultiArgs& M, int grid, int block, \
                                   size_t smem, cudaStream_t s)                                       \
    {                                                                                                 \
        return launch_multi_sx<SX>(N, words_per_thread, M, grid, block, smem, s);                     \
    }                                                                                                 \
    }

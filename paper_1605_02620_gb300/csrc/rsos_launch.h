// Host-side launch interface between the C-ABI layer and the kernels.
#pragma once
#include <cuda_runtime.h>

#include "rsos_device.cuh"
#include "rsos_gen_sched.cuh"
#include "rsos_general.cuh"
#include "rsos_persist.cuh"

namespace rsos {

// Sweep kernels, one translation unit per sub-tile edge SX in {1, 2, 4, 8}.
// Launch one phase (set q = perm[p] of sweep t) over every tile of the job.
// words_per_thread: 1 (uint32 lane words) or 2 (uint64); smem_budget: bytes of
// dynamic shared memory a block may use.
cudaError_t launch_phase(const JobDev& J, int SX, int words_per_thread, uint32_t t, int p, int q,
                         int ox, int oy, const Origin00& o, size_t smem_budget, cudaStream_t s);
cudaError_t launch_phase_plain(const JobDev& J, int SX, uint32_t t, int p, int q, int ox, int oy,
                               size_t smem_budget, cudaStream_t s);

// One phase on a (+1) tiling (section III.C): sub-tile set q = perm[p] of
// every tile of G; o locates site (0,0) in this sweep's tiling.
// *n_launches = kernels queued (1).
cudaError_t launch_phase_general(const JobDev& J, const GenTiling& G, int words_per_thread, uint32_t t, int p, int q,
                                 int ox, int oy, const GenOrigin& o, size_t smem_budget, cudaStream_t s,
                                 int* n_launches);

// Persistent engine on a (+1) tiling (rsos_gen_sched.cuh): the worker loop
// of the regular persistent engine over the tiling's rows.
constexpr int kGenPersistWarps = 3;  // warps per block
struct GenPersistArgs {
    JobDev J;
    GenTiling G;
    GenSchedGeom S;
    unsigned long long* done;      // [4][ny] completion counters
    unsigned long long* ticket;    // next ticket (zeroed before each launch)
    unsigned int* err;             // error word
    uint32_t t0;                   // first sweep of the launch
    unsigned long long n_tickets;  // items of the launch, < 2^31
    int CW, TPL;                   // tiles per item, tiles per lane
    long long budget_ns;           // time budget of every single wait
};

#define RSOS_DECLARE_SX(SX)                                                                          \
    cudaError_t launch_phase_s##SX(const JobDev& J, int words_per_thread, uint32_t t, int p, int q,  \
                                   int ox, int oy, const Origin00& o, size_t smem_budget,           \
                                   cudaStream_t s);                                                  \
    cudaError_t launch_phase_plain_s##SX(const JobDev& J, uint32_t t, int p, int q, int ox, int oy,  \
                                         size_t smem_budget, cudaStream_t s);
RSOS_DECLARE_SX(1)
RSOS_DECLARE_SX(2)
RSOS_DECLARE_SX(4)
RSOS_DECLARE_SX(8)
#undef RSOS_DECLARE_SX

// Persistent dataflow engine.  plan_persist fills the block size, chunk
// width, grid (resident blocks) and phase lag for a job; launch_persist runs
// the tickets of sweeps [A.t0, A.t0 + n) as one cooperative launch.
struct PersistPlan {
    int CW, K, D, nthr, grid;
    size_t smem;
};
// (+1) tilings: the same plan and a cooperative launch of
// general_persistent_kernel (rsos_general.cu).
cudaError_t plan_gen_persist(const JobDev& J, const GenTiling& G, int words_per_thread, int block_tiles,
                             int phase_lag, PersistPlan* out);
cudaError_t launch_gen_persist(int N, int words_per_thread, const GenPersistArgs& A, const PersistPlan& P,
                               cudaStream_t s);
// phase_lag >= 2 fixes the lag; 0 lets the plan choose it.
cudaError_t plan_persist(const JobDev& J, int SX, int words_per_thread, int block_tiles, int phase_lag,
                         PersistPlan* out);
cudaError_t launch_persist(const JobDev& J, int SX, int words_per_thread, const PersistArgs& A,
                           const PersistPlan& P, cudaStream_t s);
// 128-lane words (words_per_thread 4) on 4x4 sub-tiles, single jobs only
// (rsos_persist_w128.cu).
cudaError_t plan_persist_w128(const JobDev& J, int block_tiles, int phase_lag, PersistPlan* out);
cudaError_t launch_persist_w128(const JobDev& J, const PersistArgs& A, const PersistPlan& P, cudaStream_t s);
// Multi-job launch: all jobs share N, word width and SX.  grid from
// plan_multi (resident blocks of persistent_multi_kernel).
cudaError_t plan_multi(int N, int SX, int words_per_thread, int* grid, int* block, size_t* smem);
cudaError_t launch_multi(int N, int SX, int words_per_thread, const MultiArgs& M, int grid, int block, size_t smem,
                         cudaStream_t s);
#define RSOS_DECLARE_MULTI(SX)                                                                        \
    cudaError_t plan_multi_s##SX(int N, int words_per_thread, int* grid, int* block, size_t* smem);   \
    cudaError_t launch_multi_s##SX(int N, int words_per_thread, const MultiArgs& M, int grid, int block, \
                                   size_t smem, cudaStream_t s);
RSOS_DECLARE_MULTI(1)
RSOS_DECLARE_MULTI(2)
RSOS_DECLARE_MULTI(4)
RSOS_DECLARE_MULTI(8)
#undef RSOS_DECLARE_MULTI

#define RSOS_DECLARE_PERSIST(SX)                                                                      \
    cudaError_t plan_persist_s##SX(const JobDev& J, int words_per_thread, int block_tiles, int phase_lag, \
                                   PersistPlan* out);                                                  \
    cudaError_t launch_persist_s##SX(const JobDev& J, int words_per_thread, const PersistArgs& A,      \
                                     const PersistPlan& P, cudaStream_t s);
RSOS_DECLARE_PERSIST(1)
RSOS_DECLARE_PERSIST(2)
RSOS_DECLARE_PERSIST(4)
RSOS_DECLARE_PERSIST(8)
#undef RSOS_DECLARE_PERSIST

// Measurement (Eq. 2 numerators), exact: the 128-bit sum h and sum h^2 of
// every lane as (lo, hi) int64 pairs into rec[lane * rec_stride + 0..3]
// (partial: measure_blocks x S_pad x 2 int64).
cudaError_t launch_measure(const JobDev& J, bool plain, int S_pad, int32_t* row0, int64_t* partial,
                           int ncb_capacity, int64_t* rec, int rec_stride, cudaStream_t s);
// Power sums for the height distribution's moments: sum h^k, k = 1..4, as
// 128-bit (lo, hi) pairs into rec8[lane * 8 ...] (partial: measure_blocks x
// S_pad x 6 int64).
cudaError_t launch_moments(const JobDev& J, bool plain, int S_pad, int32_t* row0, int64_t* partial,
                           int ncb_capacity, int64_t* rec8, cudaStream_t s);
// Number of column blocks the measurement needs (partial buffer rows).
int measure_blocks(const JobDev& J, bool plain);
// Absolute heights of one lane into out[L*L] (int64).
cudaError_t launch_heights(const JobDev& J, bool plain, int lane, int32_t* row0, int64_t* out,
                           cudaStream_t s);
// Zero-fill (flat initial condition).
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s);

}  // namespace rsos

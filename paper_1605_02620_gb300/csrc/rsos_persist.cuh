// Persistent dataflow engine for the double-tiling sweep (section II).
//
// One cooperative launch runs sweeps [t0, t1) of one job with every block
// resident.  Every warp is an autonomous worker: it takes the next ticket
// (rsos_sched.cuh), waits until the items the ticket depends on are complete,
// runs the item's sub-tile activations (one lane per tile and lane-word group,
// 32 lanes = one item) and publishes the completion with a release-ordered
// counter increment, while the next ticket is already being fetched.  No
// block- or grid-wide barrier is ever taken; consecutive phases and sweeps
// overlap, and the rows between the phase-0 and phase-3 fronts stay in L2 so
// each sweep streams the lattice from HBM about once.
//
// Every wait is bounded: after kWaitIterLimit polls or the launch's time
// budget (ns, %globaltimer) a waiting block records RSOS_ETIMEOUT in the
// error word and leaves; all other blocks stop taking tickets when the error
// word is set, so the launch always ends and the context stays usable.
#pragma once
#include "rsos_device.cuh"
#include "rsos_sched.cuh"

namespace rsos {

constexpr unsigned kPersistTimeout = 1u;  // error word value for a timed-out wait

// Warps per persistent block: as many 32-lane workers (up to 4) as fit 72 KiB
// of private shared-memory windows.
RSOS_HD constexpr int persist_warps_per_block(int SX, int B, int word_bytes)
{
    return (SX + 2) * (SX + 2) * B * word_bytes * 32 * 4 <= 72 * 1024   ? 4
           : (SX + 2) * (SX + 2) * B * word_bytes * 32 * 2 <= 72 * 1024 ? 2
                                                                         : 1;
}

template <int N, typename WT, int SX>
struct PersistCfg {
    static constexpr int SLOTS = (SX + 2) * (SX + 2);  // window slots per thread
    static constexpr int WPB = persist_warps_per_block(SX, bits_for_step(N), (int)sizeof(WT));
    static constexpr int BLOCK = 32 * WPB;
    // 32- and 64-bit words: 12 warps per SM, which caps registers at ~170 per
    // thread.  128-lane words: as many blocks as their windows leave room for
    // in 227 KB of shared memory (3 blocks of 2 warps at N = 1), so the
    // register cap is the hardware's.
    static constexpr int SMEM_BLOCKS = (227 * 1024) / (SLOTS * bits_for_step(N) * (int)sizeof(WT) * BLOCK);
    static constexpr int MIN_BLOCKS = sizeof(WT) == 16 ? (SMEM_BLOCKS < 1 ? 1 : SMEM_BLOCKS) : 12 / WPB;
};

constexpr long long kWaitIterLimit = 1ll << 26;

struct PersistArgs {
    JobDev J;
    SchedGeom G;
    unsigned long long* done;     // [4][nT] completion counters (cumulative over sweeps)
    unsigned long long* ticket;   // next ticket (zeroed before each launch)
    unsigned int* err;            // error word (0 = ok)
    uint32_t t0;                  // first sweep of this launch
    unsigned long long n_tickets; // items of sweeps [t0, t1), < 2^31
    int CW;                       // tiles per chunk = TPL * (32 / NWP)
    int TPL;                      // tiles per lane and item
    long long budget_ns;          // time budget of every single wait
};

// One job of a multi-job (batch) launch: the fields of PersistArgs that
// differ between jobs.  All jobs of one launch share N, word width and tile
// edge (one kernel instantiation).
struct MultiJob {
    JobDev J;
    SchedGeom G;
    unsigned long long* done;
    unsigned long long* ticket;    // tickets handed out (zeroed before each launch)
    unsigned long long* finished;  // items completed (zeroed before each launch)
    unsigned long long n_tickets;  // < 2^31
    unsigned long long cap;        // most tickets in flight at once
    uint32_t t0;
    int CW, TPL;
    int pad_;
};

struct MultiArgs {
    const MultiJob* jobs;
    int n_jobs;
    unsigned int* first;      // lowest job index that may still have tickets (zeroed before each launch)
    unsigned int* exhausted;  // per job: 1 once its tickets ran out (zeroed before each launch)
    unsigned int* err;
    long long budget_ns;
};

#if defined(__CUDACC__)

__device__ __forceinline__ unsigned long long load_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned load_relaxed_u32(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Publish the completion of a warp's item: every lane's lattice stores are
// ordered before the counter increment (warp barrier, then a release fence
// and a relaxed add by lane 0).
__device__ __forceinline__ void publish_done(unsigned long long* counter, int lane)
{
    __syncwarp();
    if (lane == 0) {
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        asm volatile("red.relaxed.gpu.global.add.u64 [%0], 1;" ::"l"(counter) : "memory");
    }
}

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait until *p >= target.  Returns false on timeout or when another block
// reported an error.
static __device__ __noinline__ bool wait_at_least(const unsigned long long* p, unsigned long long target, const unsigned* err,
                              long long budget_ns)
{
    if (load_acquire_u64(p) >= target) return true;
    const long long deadline = global_ns() + budget_ns;
    for (long long it = 0; it < kWaitIterLimit; ++it) {
        __nanosleep(64);
        if (load_acquire_u64(p) >= target) return true;
        if ((it & 31) == 31) {
            if (load_relaxed_u32(err) != 0u) return false;
            if (global_ns() > deadline) return false;
        }
    }
    return false;
}

// One worker warp.  Lane 0 owns the ticket stream and fetches the next ticket
// while the warp works; lanes 0..3 each compute and wait on one dependency.
// The error word is read only inside waits: a warp that never waits has
// finitely many items left, and every waiting warp sees the error and stops.  An item is
// CW = TPL * 32 / NWP consecutive tiles: every lane runs TPL activations in
// turn, reusing its private window area of the warp's shared memory.
template <int N, typename WT, int SX>
__global__ void __launch_bounds__(PersistCfg<N, WT, SX>::BLOCK, PersistCfg<N, WT, SX>::MIN_BLOCKS)
    persistent_kernel(PersistArgs A)
{
    constexpr int B = bits_for_step(N);
    constexpr int T = 2 * SX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WT* sm_w = reinterpret_cast<WT*>(smem_raw) + (size_t)warp * PersistCfg<N, WT, SX>::SLOTS * B * 32;
    const int NWP = A.J.NWP;
    const int lane_tile = lane / NWP, wp = lane - lane_tile * NWP;
    const int lanes_used = (32 / NWP) * NWP;
    unsigned long long next = 0;
    if (lane == 0) next = atomicAdd(A.ticket, 1ull);
    SweepCtx sc;
    sc.t = 0xffffffffu;
    Origin00 o{};
    for (;;) {
        const unsigned long long tk = __shfl_sync(0xffffffffu, next, 0);
        if (tk >= A.n_tickets) break;
        const uint32_t t_before = sc.t;
        const Item it = item_of_ticket<T>(A.G, tk, A.t0, &sc);
        if (sc.t != t_before) o = locate_origin_site_t<T>(A.J.L, sc.ctl.ox, sc.ctl.oy);
        const Control& ctl = sc.ctl;
        Dep dep;
        int waited = 1;
        if (lane < 4 && item_dep<T>(A.G, it, lane, sc, &dep)) {
            waited = wait_at_least(A.done + (size_t)dep.p * A.G.nT + dep.r, dep.target, A.err, A.budget_ns);
            if (!waited) atomicCAS(A.err, 0u, kPersistTimeout);
        }
        if (!__all_sync(0xffffffffu, waited)) break;
        // Lanes 0..3 took the acquire loads; the warp barrier orders them
        // before every lane's staging loads (vote.sync alone is not
        // documented to order memory).
        __syncwarp();
        if (lane == 0) next = atomicAdd(A.ticket, 1ull);  // overlaps with the work below
        const int q = ctl.perm[it.p];
        if (lane < lanes_used) {
            for (int k = 0; k < A.TPL; ++k) {
                const int tx = it.c * A.CW + k * (32 / NWP) + lane_tile;
                if (tx >= A.J.nT) break;
                if (q == o.q && tx == o.tx && it.r == o.ty) {
                    activate_subtile<N, WT, SX, true, true, 32, true>(A.J, sm_w, lane, 32, tx, it.r, wp, it.t,
                                                                          it.p, q, ctl.ox, ctl.oy, o.k);
                } else {
                    activate_subtile<N, WT, SX, false, true, 32, true>(A.J, sm_w, lane, 32, tx, it.r, wp, it.t,
                                                                           it.p, q, ctl.ox, ctl.oy, -1);
                }
            }
        }
        publish_done(A.done + (size_t)it.p * A.G.nT + it.r, lane);
    }
}

// Lane 0: the next (job, ticket).  Jobs are scanned in table order from the
// lowest one not yet exhausted; a job hands out a ticket only while fewer than
// its cap are in flight (cap ~ the tickets between an item and its
// dependencies), so the warps crowd onto as few jobs as keep them busy: large
// jobs run almost alone with their rows in L2, small ones run many at a time.
// When every open job is at its cap the scan takes from the first open job.
static __device__ bool take_multi_ticket(const MultiArgs& M, int* job, unsigned long long* tk)
{
    for (int pass = 0; pass < 2; ++pass) {
        unsigned int j = *(volatile unsigned int*)M.first;
        for (; j < (unsigned int)M.n_jobs; ++j) {
            if (*(volatile unsigned int*)&M.exhausted[j]) {
                if (j == *(volatile unsigned int*)M.first) atomicMax(M.first, j + 1);
                continue;
            }
            const MultiJob& mj = M.jobs[j];
            if (pass == 0) {
                const unsigned long long issued = *(volatile unsigned long long*)mj.ticket;
                const unsigned long long fin = *(volatile unsigned long long*)mj.finished;
                if (issued >= mj.n_tickets) {
                    atomicExch(&M.exhausted[j], 1u);
                    continue;
                }
                if (issued - fin >= mj.cap) continue;
            }
            const unsigned long long t = atomicAdd(mj.ticket, 1ull);
            if (t < mj.n_tickets) {
                *job = (int)j;
                *tk = t;
                return true;
            }
            atomicExch(&M.exhausted[j], 1u);
        }
    }
    return false;
}

// Multi-job persistent engine: the single-job worker loop, with each ticket
// drawn from a job chosen round-robin among the jobs of the launch.  Jobs are
// independent, so the per-job ticket orders and completion counters keep every
// argument of the single-job engine (no deadlock, bit-identical results).
template <int N, typename WT, int SX>
__global__ void __launch_bounds__(PersistCfg<N, WT, SX>::BLOCK, PersistCfg<N, WT, SX>::MIN_BLOCKS)
    persistent_multi_kernel(MultiArgs M)
{
    constexpr int B = bits_for_step(N);
    constexpr int T = 2 * SX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WT* sm_w = reinterpret_cast<WT*>(smem_raw) + (size_t)warp * PersistCfg<N, WT, SX>::SLOTS * B * 32;
    int next_job = 0;
    unsigned long long next_tk = 0;
    int have = 0;
    SweepCtx sc;
    sc.t = 0xffffffffu;
    int sc_job = -1;
    Origin00 o{};
    if (lane == 0) have = take_multi_ticket(M, &next_job, &next_tk);
    for (;;) {
        if (!__shfl_sync(0xffffffffu, have, 0)) break;
        const int j = __shfl_sync(0xffffffffu, next_job, 0);
        const unsigned long long tk = __shfl_sync(0xffffffffu, next_tk, 0);
        const MultiJob& mj = M.jobs[j];
        JobDev J;
        J.planes = mj.J.planes;
        J.heights = nullptr;
        J.h00 = mj.J.h00;
        J.L = mj.J.L;
        J.T = T;
        J.nT = mj.J.nT;
        J.NW = mj.J.NW;
        J.NWP = mj.J.NWP;
        J.N = N;
        J.B = B;
        J.phase_order = mj.J.phase_order;
        J.seed_lo = mj.J.seed_lo;
        J.seed_hi = mj.J.seed_hi;
        J.rk = mj.J.rk;  // the job's Philox round keys, from its table entry
        const SchedGeom G = mj.G;
        const int CW = mj.CW, TPL = mj.TPL;
        if (j != sc_job) sc.t = 0xffffffffu;  // the cached sweep belongs to another job
        sc_job = j;
        const uint32_t t_before = sc.t;
        const Item it = item_of_ticket<T>(G, tk, mj.t0, &sc);
        if (sc.t != t_before) o = locate_origin_site_t<T>(J.L, sc.ctl.ox, sc.ctl.oy);
        const Control& ctl = sc.ctl;
        Dep dep;
        int waited = 1;
        if (lane < 4 && item_dep<T>(G, it, lane, sc, &dep)) {
            waited = wait_at_least(mj.done + (size_t)dep.p * G.nT + dep.r, dep.target, M.err, M.budget_ns);
            if (!waited) atomicCAS(M.err, 0u, kPersistTimeout);
        }
        if (!__all_sync(0xffffffffu, waited)) break;
        __syncwarp();  // orders lanes 0..3's acquire loads before every lane's staging
        if (lane == 0) have = take_multi_ticket(M, &next_job, &next_tk);
        const int NWP = J.NWP;
        const int lane_tile = lane / NWP, wp = lane - lane_tile * NWP;
        const int q = ctl.perm[it.p];
        if (lane < (32 / NWP) * NWP) {
            for (int k = 0; k < TPL; ++k) {
                const int tx = it.c * CW + k * (32 / NWP) + lane_tile;
                if (tx >= J.nT) break;
                if (q == o.q && tx == o.tx && it.r == o.ty) {
                    activate_subtile<N, WT, SX, true, true, 32, true>(J, sm_w, lane, 32, tx, it.r, wp, it.t,
                                                                           it.p, q, ctl.ox, ctl.oy, o.k);
                } else {
                    activate_subtile<N, WT, SX, false, true, 32, true>(J, sm_w, lane, 32, tx, it.r, wp, it.t,
                                                                            it.p, q, ctl.ox, ctl.oy, -1);
                }
            }
        }
        publish_done(mj.done + (size_t)it.p * G.nT + it.r, lane);
        if (lane == 0) atomicAdd(mj.finished, 1ull);
    }
}

#endif  // __CUDACC__

}  // namespace rsos

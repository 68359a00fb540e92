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
    static constexpr int WPB = persist_warps_per_block(SX, bits_for_step(N), (int)sizeof(WT));
    static constexpr int BLOCK = 32 * WPB;
};

constexpr long long kWaitIterLimit = 1ll << 26;

struct PersistArgs {
    JobDev J;
    SchedGeom G;
    const uint32_t* table;        // order table, 4 * nT * K entries
    unsigned long long* done;     // [4][nT] completion counters (cumulative over sweeps)
    unsigned long long* ticket;   // next ticket (zeroed before each launch)
    unsigned int* err;            // error word (0 = ok)
    uint32_t t0;                  // first sweep of this launch
    unsigned long long n_tickets; // items of sweeps [t0, t1), < 2^31
    int CW;                       // tiles per chunk = TPL * (32 / NWP)
    int TPL;                      // tiles per lane and item
    long long budget_ns;          // time budget of every single wait
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
// while the warp works; lanes 0..3 each wait on one dependency.  An item is
// CW = TPL * 32 / NWP consecutive tiles: every lane runs TPL activations in
// turn, reusing its private window area of the warp's shared memory.
template <int N, typename WT, int SX>
__global__ void __launch_bounds__(PersistCfg<N, WT, SX>::BLOCK)
    persistent_kernel(PersistArgs A)
{
    constexpr int B = bits_for_step(N);
    constexpr int T = 2 * SX;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WT* sm_w = reinterpret_cast<WT*>(smem_raw) + (size_t)warp * (SX + 2) * (SX + 2) * B * 32;
    const int NWP = A.J.NWP;
    const int lane_tile = lane / NWP, wp = lane - lane_tile * NWP;
    const int lanes_used = (32 / NWP) * NWP;
    unsigned long long next = 0;
    if (lane == 0) next = atomicAdd(A.ticket, 1ull);
    for (;;) {
        const unsigned long long tk = __shfl_sync(0xffffffffu, next, 0);
        int ok = tk < A.n_tickets;
        if (lane == 0 && ok) ok = load_relaxed_u32(A.err) == 0u;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) break;
        const Item it = item_of_ticket<T>(A.G, A.table, tk, A.t0);
        Dep d[4];
        const int nd = item_deps<T>(A.G, it, d);
        int waited = 1;
        if (lane < nd) {
            waited = wait_at_least(A.done + (size_t)d[lane].p * A.G.nT + d[lane].r, d[lane].target, A.err,
                                   A.budget_ns);
            if (!waited) atomicCAS(A.err, 0u, kPersistTimeout);
        }
        if (!__all_sync(0xffffffffu, waited)) break;
        if (lane == 0) next = atomicAdd(A.ticket, 1ull);  // overlaps with the work below
        const Control ctl = sweep_control(A.J.seed_lo, A.J.seed_hi, it.t, T, T, A.J.phase_order);
        const int q = ctl.perm[it.p];
        const Origin00 o = locate_origin_site_t<T>(A.J.L, ctl.ox, ctl.oy);
        if (lane < lanes_used) {
            for (int k = 0; k < A.TPL; ++k) {
                const int tx = it.c * A.CW + k * (32 / NWP) + lane_tile;
                if (tx >= A.J.nT) break;
                if (q == o.q && tx == o.tx && it.r == o.ty) {
                    activate_subtile<N, WT, SX, true, true, 32>(A.J, sm_w, lane, 32, tx, it.r, wp, it.t, it.p, q,
                                                                ctl.ox, ctl.oy, o.k);
                } else {
                    activate_subtile<N, WT, SX, false, true, 32>(A.J, sm_w, lane, 32, tx, it.r, wp, it.t, it.p, q,
                                                                 ctl.ox, ctl.oy, -1);
                }
            }
        }
        __threadfence();  // the warp's lattice stores, visible GPU-wide before the release
        __syncwarp();
        if (lane == 0) atomicAdd(A.done + (size_t)it.p * A.G.nT + it.r, 1ull);
    }
}

#endif  // __CUDACC__

}  // namespace rsos

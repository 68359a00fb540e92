// Phase kernel of the double-tiling sweep on the (+1) tilings of the
// decomposition check (section III.C): one launch activates sub-tile set
// q = perm[p] of every tile, one thread per (tile, lane-word group), as the
// regular phase kernel does, with the tile and sub-tile extents taken at run
// time (T or T + 1 wide tiles, halves of floor(w/2) and the rest), over the
// class-interleaved site records of the regular tiling (column classes of
// the x base edge).  Each
// selection is Eq. 6 on bit-sliced words; the stream is the regular one with
// a = the sub-tile's own area: 2a selections per activation, site index
// k = floor(u a / 2^16) of a 16-bit u, kx = k mod w, ky = k div w.
#include <mutex>

#include "rsos_gen_sched.cuh"
#include "rsos_general.cuh"
#include "rsos_launch.h"

namespace rsos {

namespace {

template <int N, typename WT, bool HAS00>
__device__ __forceinline__ void general_activate(const JobDev& J, const GenTiling& G, WT* __restrict__ sm, int tid,
                                                 int nthr, int tx, int ty, int wp, uint32_t t, int p, int q, int ox,
                                                 int oy, int k00)
{
    constexpr int B = bits_for_step(N);
    constexpr int NWT = (int)(sizeof(WT) / 4);
    const int qx = q & 1, qy = q >> 1;
    const int w0 = wp * NWT;
    const int L = J.L;
    int u0, sw, v0, sh;
    gen_half(G.x, tx, qx, u0, sw);
    gen_half(G.y, ty, qy, v0, sh);
    const int WW = sw + 2;
    const size_t rec_words = (size_t)B * J.NW;
    const bool whole_record = NWT == J.NW;
    const size_t rs = (size_t)nthr * B;  // one slot

    // Stage the sub-tile and its one-site halo (corners unused), column by
    // column: window column ii is lattice column ox + u0 + ii - 1.
    GenCol col = gen_col(L, J.T, ox + u0 - 1);
    for (int ii = 0; ii < sw + 2; ++ii) {
        const size_t cw = gen_col_words(col, J.nT, rec_words) + (size_t)w0;
        const bool edge_col = ii == 0 || ii == sw + 1;
        for (int jj = edge_col ? 1 : 0; jj < (edge_col ? sh + 1 : sh + 2); ++jj) {
            WT* slot = sm + ((size_t)(jj * WW + ii) * nthr + tid) * B;
            const size_t rw = gen_row_words(L, J.T, J.nT, rec_words, oy + v0 + jj - 1);
            if (!RSOS_CHECK_GLOBAL(J, J.planes + rw + cw, (size_t)(B - 1) * J.NW + NWT) ||
                !RSOS_CHECK_SHARED(J, slot, sizeof(WT) * B))
                continue;
            stage_record_async<WT, B>(slot, J.planes + rw + cw, J.NW, whole_record);
        }
        gen_col_next(col, L, J.T);
    }
    stage_wait_all();

    const uint32_t tile_id = (uint32_t)(ty * G.x.n + tx);
    const uint32_t A = (uint32_t)(sw * sh);
    const int NSEL = 2 * (int)A;
    const uint32_t inv = gen_inv((uint32_t)sw);
    const uint32_t pbits = (uint32_t)p << 28;
#pragma unroll 1
    for (int g8 = 0; g8 < (NSEL + 7) / 8; ++g8) {
        const U4 site_r = philox4x32_10(U4{tile_id, t, (uint32_t)g8, kDomSite | pbits}, J.rk);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int g = 2 * g8 + h;
            if (4 * g >= NSEL) break;
            const U4 m_lo = philox4x32_10(U4{tile_id, t, (uint32_t)g, kDomMask | pbits | (uint32_t)w0}, J.rk);
            U4 m_hi = m_lo;
            if (NWT == 2) m_hi = philox4x32_10(U4{tile_id, t, (uint32_t)g, kDomMask | pbits | (uint32_t)(w0 + 1)}, J.rk);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i8 = 4 * h + r;
                if (8 * g8 + i8 >= NSEL) break;
                const uint32_t word = pick_word(site_r, i8 >> 1);
                const uint32_t half = (i8 & 1) ? (word >> 16) : (word & 0xFFFFu);
                const uint32_t k = (half * A) >> 16;
                const uint32_t ky = gen_div(k, inv);
                const uint32_t kx = k - ky * (uint32_t)sw;
                const int s = ((int)ky + 1) * WW + (int)kx + 1;
                WT* base = sm + ((size_t)s * nthr + tid) * B;
                if (!RSOS_CHECK_SHARED(J, base - (size_t)WW * rs, sizeof(WT) * B) ||
                    !RSOS_CHECK_SHARED(J, base + (size_t)WW * rs, sizeof(WT) * B))
                    continue;
                WT x[B], e[B], w[B], n[B], so[B];
                load_rec<B, WT>(base, x);
                load_rec<B, WT>(base + rs, e);
                load_rec<B, WT>(base - rs, w);
                load_rec<B, WT>(base - (size_t)WW * rs, n);
                load_rec<B, WT>(base + (size_t)WW * rs, so);
                const WT acc = accept_mask<N, B, WT>(mask_word<WT>(m_lo, m_hi, r), x, e, w, n, so);
                masked_increment<B, WT>(x, acc);
                store_rec<B, WT>(base, x);
                if (HAS00 && (int)k == k00) record_origin_deposits<WT>(J.h00, w0 * 32, acc);
            }
        }
    }

    // Write the interior back.
    col = gen_col(L, J.T, ox + u0);
    for (int ii = 1; ii <= sw; ++ii) {
        const size_t cw = gen_col_words(col, J.nT, rec_words) + (size_t)w0;
        gen_col_next(col, L, J.T);
        for (int jj = 1; jj <= sh; ++jj) {
            const WT* slot = sm + ((size_t)(jj * WW + ii) * nthr + tid) * B;
            uint32_t* dst = J.planes + gen_row_words(L, J.T, J.nT, rec_words, oy + v0 + jj - 1) + cw;
            if (!RSOS_CHECK_GLOBAL(J, dst, (size_t)(B - 1) * J.NW + NWT) || !RSOS_CHECK_SHARED(J, slot, sizeof(WT) * B))
                continue;
            WT v[B];
            load_rec<B, WT>(slot, v);
            if (B * sizeof(WT) == 16 && whole_record) {
                if (sizeof(WT) == 8)
                    *reinterpret_cast<ulonglong2*>(dst) =
                        make_ulonglong2((unsigned long long)v[0], (unsigned long long)v[B - 1]);
                else
                    *reinterpret_cast<uint4*>(dst) =
                        make_uint4((unsigned)v[0], (unsigned)v[1 % B], (unsigned)v[2 % B], (unsigned)v[B - 1]);
            } else {
#pragma unroll
                for (int b = 0; b < B; ++b) *reinterpret_cast<WT*>(dst + (size_t)b * J.NW) = v[b];
            }
        }
    }
}

template <int N, typename WT>
__global__ void __launch_bounds__(256) general_phase_kernel(JobDev J, GenTiling G, GenLaunch P, uint32_t t, int p,
                                                            int q, int ox, int oy, GenOrigin o)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WT* sm = reinterpret_cast<WT*>(smem_raw);
    const int tid = threadIdx.x;
    int tx, ty, wp, nthr;
    if (!gen_item_of_thread(P, J.NWP, (int)blockIdx.x, tid, (int)blockDim.x, tx, ty, wp, nthr)) return;
    if (q == o.q && tx == o.tx && ty == o.ty)
        general_activate<N, WT, true>(J, G, sm, tid, nthr, tx, ty, wp, t, p, q, ox, oy, o.k);
    else
        general_activate<N, WT, false>(J, G, sm, tid, nthr, tx, ty, wp, t, p, q, ox, oy, -1);
}

// Persistent dataflow engine on a (+1) tiling: the worker loop of the
// regular persistent engine (rsos_persist.cuh) over the items and
// dependencies of rsos_gen_sched.cuh, each lane activating its tile's
// sub-tile with the extents of that tile (general_activate).  Every warp owns
// windows for the widest half of either axis.
template <int N, typename WT>
__global__ void __launch_bounds__(32 * kGenPersistWarps, 4) general_persistent_kernel(GenPersistArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int B = bits_for_step(N);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t slots = (size_t)(A.G.max_w + 2) * (size_t)(A.G.max_h + 2);
    WT* sm_w = reinterpret_cast<WT*>(smem_raw) + (size_t)warp * slots * B * 32;
    const int NWP = A.J.NWP;
    const int lane_tile = lane / NWP, wp = lane - lane_tile * NWP;
    const int lanes_used = (32 / NWP) * NWP;
    const int ny = A.S.y.n;
    unsigned long long next = 0;
    if (lane == 0) next = atomicAdd(A.ticket, 1ull);
    GenSweepCtx sc;
    sc.t = 0xffffffffu;
    GenOrigin o{};
    for (;;) {
        const unsigned long long tk = __shfl_sync(0xffffffffu, next, 0);
        if (tk >= A.n_tickets) break;
        const uint32_t t_before = sc.t;
        const Item it = gen_item_of_ticket(A.S, tk, A.t0, &sc);
        if (sc.t != t_before) o = gen_locate_origin_site(A.J.L, A.G, sc.ctl.ox, sc.ctl.oy);
        Dep dep;
        int waited = 1;
        if (lane < 4 && gen_item_dep(A.S, it, lane, sc, &dep)) {
            waited = wait_at_least(A.done + (size_t)dep.p * ny + dep.r, dep.target, A.err, A.budget_ns);
            if (!waited) atomicCAS(A.err, 0u, kPersistTimeout);
        }
        if (!__all_sync(0xffffffffu, waited)) break;
        __syncwarp();  // orders lanes 0..3's acquire loads before every lane's staging
        if (lane == 0) next = atomicAdd(A.ticket, 1ull);  // overlaps with the work below
        const int q = sc.ctl.perm[it.p];
        if (lane < lanes_used) {
            for (int k = 0; k < A.TPL; ++k) {
                const int tx = it.c * A.CW + k * (32 / NWP) + lane_tile;
                if (tx >= A.G.x.n) break;
                if (q == o.q && tx == o.tx && it.r == o.ty)
                    general_activate<N, WT, true>(A.J, A.G, sm_w, lane, 32, tx, it.r, wp, it.t, it.p, q, sc.ctl.ox,
                                                  sc.ctl.oy, o.k);
                else
                    general_activate<N, WT, false>(A.J, A.G, sm_w, lane, 32, tx, it.r, wp, it.t, it.p, q, sc.ctl.ox,
                                                   sc.ctl.oy, -1);
            }
        }
        publish_done(A.done + (size_t)it.p * ny + it.r, lane);
    }
}

constexpr size_t kMaxDynamicSmem = 227 * 1024;  // largest dynamic shared memory of a block

// Allows general_phase_kernel<N, WT> the largest dynamic shared memory, once
// (thread-safe static initialisation).
template <int N, typename WT>
cudaError_t general_allow_smem()
{
    static const cudaError_t e = cudaFuncSetAttribute(general_phase_kernel<N, WT>,
                                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                      (int)kMaxDynamicSmem);
    return e;
}

// Threads per block that keep the most threads resident per SM for windows
// of per_thread bytes (shared memory is the limit; ties go to larger blocks).
template <int N, typename WT>
int general_block_threads(size_t per_thread, size_t smem_cap)
{
    int best = 32, best_resident = -1;
    for (int n = 32; n <= 256; n += 32) {
        const size_t smem = per_thread * (size_t)n;
        if (smem > smem_cap) break;
        int blocks = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, general_phase_kernel<N, WT>, n, smem) !=
            cudaSuccess) {
            (void)cudaGetLastError();
            break;
        }
        if (blocks * n >= best_resident) {
            best_resident = blocks * n;
            best = n;
        }
    }
    return best;
}

template <int N, typename WT>
cudaError_t launch_general_t(const JobDev& J, const GenTiling& G, uint32_t t, int p, int q, int ox, int oy,
                             const GenOrigin& o, size_t smem_budget, cudaStream_t s, int* n_launches)
{
    constexpr int B = bits_for_step(N);
    *n_launches = 0;
    const size_t wbytes = (size_t)B * sizeof(WT);  // one window slot
    const size_t pt_narrow = gen_narrow_window_slots(G) * wbytes;
    const size_t pt_wide = (size_t)(G.max_w + 2) * (G.max_h + 2) * wbytes;
    if (pt_wide * 8 > kMaxDynamicSmem) return cudaErrorInvalidConfiguration;
    const cudaError_t allowed = general_allow_smem<N, WT>();
    if (allowed != cudaSuccess) return allowed;
    const size_t cap = smem_budget < pt_narrow * 32 ? pt_narrow * 32 : smem_budget;
    // block size per (window bytes, budget), remembered for a few windows;
    // handles on different host threads may launch concurrently
    struct Plan {
        size_t per_thread, cap;
        int n;
    };
    static Plan plans[8] = {};
    static int n_plans = 0;
    static std::mutex plans_mu;
    int n = 0;
    {
        std::lock_guard<std::mutex> lock(plans_mu);
        for (int k = 0; k < n_plans; ++k)
            if (plans[k].per_thread == pt_narrow && plans[k].cap == cap) n = plans[k].n;
    }
    if (n == 0) {
        n = general_block_threads<N, WT>(pt_narrow, cap > kMaxDynamicSmem ? kMaxDynamicSmem : cap);
        std::lock_guard<std::mutex> lock(plans_mu);
        if (n_plans < 8) plans[n_plans++] = Plan{pt_narrow, cap, n};
    }
    GenLaunch P;
    size_t smem = 0;
    long long blocks = 0;
    gen_plan_launch(G, J.NWP, wbytes, n, P, smem, blocks);
    if (blocks == 0) return cudaSuccess;
    general_phase_kernel<N, WT><<<(unsigned)blocks, (unsigned)n, smem, s>>>(J, G, P, t, p, q, ox, oy, o);
    *n_launches = 1;
    return cudaGetLastError();
}

template <int N, typename WT>
cudaError_t plan_gen_persist_t(const JobDev& J, const GenTiling& G, int block_tiles, int phase_lag, PersistPlan* P)
{
    constexpr int B = bits_for_step(N);
    const size_t per_thread = (size_t)(G.max_w + 2) * (size_t)(G.max_h + 2) * B * sizeof(WT);
    P->CW = block_tiles;
    if (P->CW < 1) return cudaErrorInvalidConfiguration;
    P->K = (G.x.n + P->CW - 1) / P->CW;
    P->nthr = 32 * kGenPersistWarps;
    P->smem = per_thread * (size_t)P->nthr;
    if (P->smem > kMaxDynamicSmem) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(general_persistent_kernel<N, WT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)P->smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, general_persistent_kernel<N, WT>, P->nthr, P->smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    P->grid = per_sm * sms;
    // phase lag as for the regular engine: 1.5 x the items in flight (two
    // per worker warp) per slot of 4K items, at most a third of the rows
    const int per_slot = 4 * P->K;
    const int workers = P->grid * kGenPersistWarps;
    int D = (int)(1.5 * 2.0 * workers / per_slot);
    const int dmax = G.y.n / 3 > 2 ? G.y.n / 3 : 2;
    if (D > dmax) D = dmax;
    if (D < 2) D = 2;
    if (phase_lag >= 2) D = phase_lag;
    P->D = D;
    (void)J;
    return cudaSuccess;
}

template <int N, typename WT>
cudaError_t launch_gen_persist_t(const GenPersistArgs& A, const PersistPlan& P, cudaStream_t s)
{
    GenPersistArgs a = A;
    void* args[] = {&a};
    return cudaLaunchCooperativeKernel((const void*)general_persistent_kernel<N, WT>, dim3(P.grid), dim3(P.nthr), args,
                                       P.smem, s);
}

}  // namespace

cudaError_t plan_gen_persist(const JobDev& J, const GenTiling& G, int words_per_thread, int block_tiles,
                             int phase_lag, PersistPlan* out)
{
#define RSOS_CASE(NN)                                                                                     \
    case NN:                                                                                              \
        return words_per_thread == 2 ? plan_gen_persist_t<NN, uint64_t>(J, G, block_tiles, phase_lag, out) \
                                     : plan_gen_persist_t<NN, uint32_t>(J, G, block_tiles, phase_lag, out);
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

cudaError_t launch_gen_persist(int N, int words_per_thread, const GenPersistArgs& A, const PersistPlan& P,
                               cudaStream_t s)
{
#define RSOS_CASE(NN)                                                                   \
    case NN:                                                                            \
        return words_per_thread == 2 ? launch_gen_persist_t<NN, uint64_t>(A, P, s)      \
                                     : launch_gen_persist_t<NN, uint32_t>(A, P, s);
    switch (N) {
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

cudaError_t launch_phase_general(const JobDev& J, const GenTiling& G, int words_per_thread, uint32_t t, int p, int q,
                                 int ox, int oy, const GenOrigin& o, size_t smem_budget, cudaStream_t s,
                                 int* n_launches)
{
#define RSOS_CASE(NN)                                                                                      \
    case NN:                                                                                               \
        return words_per_thread == 2                                                                       \
                   ? launch_general_t<NN, uint64_t>(J, G, t, p, q, ox, oy, o, smem_budget, s, n_launches) \
                   : launch_general_t<NN, uint32_t>(J, G, t, p, q, ox, oy, o, smem_budget, s, n_launches);
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

}  // namespace rsos

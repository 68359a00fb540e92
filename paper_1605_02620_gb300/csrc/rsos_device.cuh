// Device-side data structures and the sub-tile activation of the RSOS
// double-tiling sweep (section II of the paper; Eq. 6 for the update rule).
//
// Data layout in HBM (multisurface path).  A job of S surfaces has
// NW = ceil(S/32) lane words; bit j of word w is surface 32*w + j.  The
// residue h mod 2^B of every site is stored in B bit planes.  Sites are
// ordered  [y][x mod T][x div T]  ("class-interleaved" by the tile edge T):
// the same column class of consecutive tiles is contiguous, so a warp whose
// threads work on consecutive tiles reads and writes one contiguous run
// whatever the random tiling origin of the sweep is.  Each site is one
// record of B planes x NW words (plane-major inside the record): for 64
// surfaces and N = 1 a record is 16 bytes, so one 16-byte copy moves a
// site and every record starts on a 16-byte boundary.
//
// Shared memory (per thread, private): the active sub-tile plus its one-site
// halo, (SX+2) x (SY+2) slots (corners unused), each slot one record of the
// thread's lane-word group, stored [slot][thread][plane]: consecutive
// threads own consecutive records, so random per-thread site choices never
// conflict and a record is one vector access.
#pragma once
#include "philox.cuh"
#include "rsos_logic.cuh"

namespace rsos {

struct JobDev {
    uint32_t* planes;   // multisurface: L*L site records of B planes x NW words
    int32_t* heights;   // plain path: L*L int32, row-major
    int64_t* h00;       // absolute height of site (0,0) per lane (NW*32)
    int32_t L, T, nT;   // lattice edge, tile edge (square tiles), tiles per row
    int32_t NW;         // 32-lane words per site and plane
    int32_t NWP;        // thread groups per tile (NW / words per thread)
    int32_t N, B;
    int32_t phase_order;
    uint32_t seed_lo, seed_hi;
    RoundKeys rk;       // Philox round keys of the seed
    uint32_t* bounds_err;  // checked build: count of out-of-range accesses (nullable)
};

// Where site (0,0) lies in the tiling of one sweep.
struct Origin00 {
    int tx, ty;  // tile
    int q;       // sub-tile set
    int k;       // site index inside the sub-tile
};

RSOS_HD Origin00 locate_origin_site(int L, int T, int ox, int oy)
{
    const int S = T / 2;
    const int xr = ox == 0 ? 0 : L - ox, yr = oy == 0 ? 0 : L - oy;
    Origin00 o;
    o.tx = xr / T;
    o.ty = yr / T;
    const int u = xr - o.tx * T, v = yr - o.ty * T;
    o.q = 2 * (v >= S ? 1 : 0) + (u >= S ? 1 : 0);
    o.k = (v >= S ? v - S : v) * S + (u >= S ? u - S : u);
    return o;
}

// Same with the tile edge known at compile time (shifts instead of divisions).
template <int T>
RSOS_HD Origin00 locate_origin_site_t(int L, int ox, int oy)
{
    return locate_origin_site(L, T, ox, oy);
}

// Index of the record of site (x, y).
RSOS_HD size_t site_record(const JobDev& J, int x, int y)
{
    return ((size_t)y * J.T + (size_t)(x % J.T)) * J.nT + (size_t)(x / J.T);
}

// Word offset of plane b, lane word w of record rec.
RSOS_HD size_t plane_word(const JobDev& J, size_t rec, int b, int w)
{
    return (rec * (size_t)J.B + (size_t)b) * (size_t)J.NW + (size_t)w;
}

// Word offsets (plane 0, lane word w0) of the window columns i = -1..SX and
// rows j = -1..SY of the active sub-tile of tile (tx, ty) in the sweep's
// tiling; plane b is b * NW words further.
template <int SX>
struct WindowIndex {
    size_t col[SX + 2];
    size_t row[SX + 2];
};

template <int SX>
RSOS_HD void window_index(const JobDev& J, int tx, int ty, int qx, int qy, int ox,
                                             int oy, int w0, WindowIndex<SX>& wi)
{
    constexpr int T = 2 * SX;  // square tiles: the tile edge is known at compile time
    const int nT = J.nT, L = J.L;
    const size_t rec_words = (size_t)J.B * J.NW;
#pragma unroll
    for (int ii = 0; ii < SX + 2; ++ii) {
        int xr = ox + qx * SX + ii - 1;  // in [-1, 2T)
        int dm = 0;
        if (xr < 0) {
            xr += T;
            dm = -1;
        } else if (xr >= T) {
            xr -= T;
            dm = 1;
        }
        int col = tx + dm;
        col = col < 0 ? col + nT : (col >= nT ? col - nT : col);
        wi.col[ii] = ((size_t)xr * nT + col) * rec_words + w0;
    }
#pragma unroll
    for (int jj = 0; jj < SX + 2; ++jj) {
        int y = oy + ty * T + qy * SX + jj - 1;  // in [-1, L + T)
        y = y < 0 ? y + L : (y >= L ? y - L : y);
        wi.row[jj] = (size_t)y * ((size_t)T * nT * rec_words);
    }
}

#if defined(__CUDACC__)

// Checked build (RSOS_CHECKED): every record a sweep kernel stages or writes
// back is tested against the lattice, and every shared-memory record it
// touches against the block's dynamic shared memory.  A failed test counts
// in *J.bounds_err and the access is skipped (no trap: the context stays
// usable).  In the normal build both tests are the constant true.
#if defined(RSOS_CHECKED)
__device__ __forceinline__ void count_bounds_error(const JobDev& J)
{
    if (J.bounds_err) atomicAdd(J.bounds_err, 1u);
}

// words 32-bit words from p lie inside the multisurface lattice.
__device__ __forceinline__ bool check_global(const JobDev& J, const uint32_t* p, size_t words)
{
    const size_t total = (size_t)J.B * (size_t)J.L * (size_t)J.T * (size_t)J.nT * (size_t)J.NW;
    const bool ok = p >= J.planes && (size_t)(p - J.planes) + words <= total;
    if (!ok) count_bounds_error(J);
    return ok;
}

// bytes bytes from p lie inside the block's dynamic shared memory.
__device__ __forceinline__ bool check_shared(const JobDev& J, const void* p, size_t bytes)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned dyn = 0;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const unsigned char* c = static_cast<const unsigned char*>(p);
    const bool ok = c >= smem_raw && (size_t)(c - smem_raw) + bytes <= (size_t)dyn;
    if (!ok) count_bounds_error(J);
    return ok;
}
#define RSOS_CHECK_GLOBAL(J, p, words) ::rsos::check_global((J), (p), (words))
#define RSOS_CHECK_SHARED(J, p, bytes) ::rsos::check_shared((J), (p), (bytes))
#else
#define RSOS_CHECK_GLOBAL(J, p, words) true
#define RSOS_CHECK_SHARED(J, p, bytes) true
#endif

template <typename WT>
__device__ __forceinline__ WT mask_word(const U4& lo, const U4& hi, int r);

template <>
__device__ __forceinline__ uint32_t mask_word<uint32_t>(const U4& lo, const U4&, int r)
{
    return r == 0 ? lo.x : r == 1 ? lo.y : r == 2 ? lo.z : lo.w;
}

template <>
__device__ __forceinline__ uint64_t mask_word<uint64_t>(const U4& lo, const U4& hi, int r)
{
    const uint32_t a = r == 0 ? lo.x : r == 1 ? lo.y : r == 2 ? lo.z : lo.w;
    const uint32_t b = r == 0 ? hi.x : r == 1 ? hi.y : r == 2 ? hi.z : hi.w;
    return (uint64_t)a | ((uint64_t)b << 32);
}

__device__ __forceinline__ uint32_t pick_word(const U4& v, int r)
{
    return r == 0 ? v.x : r == 1 ? v.y : r == 2 ? v.z : v.w;
}

// Deposits accepted at site (0,0) raise its tracked absolute height.  Atomic
// so that blocks of a persistent launch never see a stale cached value.
template <typename WT>
__device__ __forceinline__ void record_origin_deposits(int64_t* h00, int lane_base, WT acc)
{
    while (acc) {
        const int bit = sizeof(WT) == 8 ? __ffsll((long long)acc) - 1 : __ffs((int)acc) - 1;
        atomicAdd(reinterpret_cast<unsigned long long*>(h00 + lane_base + bit), 1ull);
        acc &= acc - 1;
    }
}

template <>
__device__ __forceinline__ void record_origin_deposits<Word128>(int64_t* h00, int lane_base, Word128 acc)
{
    record_origin_deposits<unsigned long long>(h00, lane_base, acc.lo);
    record_origin_deposits<unsigned long long>(h00, lane_base + 64, acc.hi);
}

// Plain global load of one lattice word (phase-by-phase engine: every phase is
// its own launch, so no other block writes the lattice meanwhile).
template <typename WT>
__device__ __forceinline__ WT load_word(const uint32_t* p)
{
    return *reinterpret_cast<const WT*>(p);
}

// Asynchronous copy of this thread's part of one site record into its
// shared-memory slot (global -> shared without a register round trip, so all
// copies of a window are in flight at once).  When the thread owns whole
// records of a size that is a multiple of 16 bytes (64 surfaces, N = 1: 16 B)
// they move as 16-byte copies that bypass L1; otherwise plane by plane
// through L1, which the persistent engines keep coherent by the acquire load
// they take before every item.
//   dst   slot in shared memory (B words of WT)
//   src   plane-0 word of the thread's lane-word group in the record
template <typename WT, int B>
__device__ __forceinline__ void stage_record_async(WT* dst, const uint32_t* src, int NW, bool whole_record)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    constexpr int bytes = B * (int)sizeof(WT);
    if (bytes % 16 == 0 && whole_record) {
#pragma unroll
        for (int c = 0; c < bytes / 16; ++c)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16 * c), "l"(src + 4 * c) : "memory");
        return;
    }
    // A whole record of 8 bytes (two planes of one 32-lane word; records are
    // 8-byte aligned): one 8-byte copy instead of one per plane (2% faster
    // sweeps at N = 1 with 32 surfaces).
    if (bytes == 8 && whole_record) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
        return;
    }

#pragma unroll
    for (int b = 0; b < B; ++b) {
        if (sizeof(WT) == 16)  // 128-lane words: 16-byte aligned, bypass L1
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + 16 * b), "l"(src + (size_t)b * NW)
                         : "memory");
        else if (sizeof(WT) == 8)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d + 8 * b), "l"(src + (size_t)b * NW)
                         : "memory");
        else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d + 4 * b), "l"(src + (size_t)b * NW)
                         : "memory");
    }
}

// Wait for this thread's outstanding asynchronous copies.
__device__ __forceinline__ void stage_wait_all()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// One record (B words) of a shared-memory slot, as vector accesses where the
// size allows (16-byte aligned: slots are B * sizeof(WT) bytes apart).
template <int B, typename WT>
__device__ __forceinline__ void load_rec(const WT* p, WT (&v)[B])
{
    if constexpr (B * sizeof(WT) == 16) {
        if constexpr (sizeof(WT) == 8) {
            const ulonglong2 q = *reinterpret_cast<const ulonglong2*>(p);
            v[0] = (WT)q.x;
            v[B - 1] = (WT)q.y;
        } else {
            const uint4 q = *reinterpret_cast<const uint4*>(p);
            v[0] = (WT)q.x;
            v[1 % B] = (WT)q.y;
            v[2 % B] = (WT)q.z;
            v[B - 1] = (WT)q.w;
        }
    } else if constexpr (B * sizeof(WT) == 32 && sizeof(WT) == 8) {
        const ulonglong2 q0 = *reinterpret_cast<const ulonglong2*>(p);
        const ulonglong2 q1 = *reinterpret_cast<const ulonglong2*>(p + 2);
        v[0] = (WT)q0.x;
        v[1 % B] = (WT)q0.y;
        v[2 % B] = (WT)q1.x;
        v[B - 1] = (WT)q1.y;
    } else {
#pragma unroll
        for (int b = 0; b < B; ++b) v[b] = p[b];
    }
}

template <int B, typename WT>
__device__ __forceinline__ void store_rec(WT* p, const WT (&v)[B])
{
    if constexpr (B * sizeof(WT) == 16) {
        if constexpr (sizeof(WT) == 8) {
            *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2((unsigned long long)v[0], (unsigned long long)v[B - 1]);
        } else {
            *reinterpret_cast<uint4*>(p) =
                make_uint4((unsigned)v[0], (unsigned)v[1 % B], (unsigned)v[2 % B], (unsigned)v[B - 1]);
        }
    } else if constexpr (B * sizeof(WT) == 32 && sizeof(WT) == 8) {
        *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2((unsigned long long)v[0], (unsigned long long)v[1 % B]);
        *reinterpret_cast<ulonglong2*>(p + 2) =
            make_ulonglong2((unsigned long long)v[2 % B], (unsigned long long)v[B - 1]);
    } else {
#pragma unroll
        for (int b = 0; b < B; ++b) p[b] = v[b];
    }
}

// Write-back of a whole 16-byte record (slot -> lattice) as one vector store;
// compiled only for the word types whose records are 16 bytes.
template <int B, typename WT>
__device__ __forceinline__ void store_record16(uint32_t* dst, const WT* slot)
{
    if constexpr (B * sizeof(WT) == 16) {
        WT v[B];
        load_rec<B, WT>(slot, v);
        if constexpr (sizeof(WT) == 8)
            *reinterpret_cast<ulonglong2*>(dst) = make_ulonglong2((unsigned long long)v[0], (unsigned long long)v[B - 1]);
        else
            *reinterpret_cast<uint4*>(dst) =
                make_uint4((unsigned)v[0], (unsigned)v[1 % B], (unsigned)v[2 % B], (unsigned)v[B - 1]);
    }
}

// The 2a selections of one sub-tile activation (section II; Eq. 6 per
// selection) on a window already staged in shared memory: slot s of this
// thread at sm[((s * nthr) + tid) * B], (SX+2)^2 slots row-major with the
// sub-tile at rows and columns 1..SX.
//   tile_id   tile index of the Philox counters;  w0  first lane word
//   k00       site index of global site (0,0) in this sub-tile (HAS00)
template <int N, typename WT, int SX, bool HAS00, int NTHR = 0, bool RKEYS = true>
__device__ __forceinline__ void select_subtile(const JobDev& J, WT* __restrict__ sm, int tid, int nthr_rt,
                                               uint32_t tile_id, uint32_t t, int p, int w0, int k00)
{
    const int nthr = NTHR > 0 ? NTHR : nthr_rt;
    constexpr int B = bits_for_step(N);
    constexpr int A = SX * SX;
    constexpr int NSEL = 2 * A;
    constexpr int WW = SX + 2;
    constexpr int NWT = (int)(sizeof(WT) / 4);
    const uint32_t pbits = (uint32_t)p << 28;
    // Eight selections per site draw (16-bit halves), four per mask draw; the
    // blocks of eight are unrolled so every word index is static.
#pragma unroll 1
    for (int g8 = 0; g8 < (NSEL + 7) / 8; ++g8) {
        // RKEYS: round keys from the job descriptor; else derived from the seed
        // (jobs of a batch read their descriptor from global memory).
        const U4 site_r = RKEYS ? philox4x32_10(U4{tile_id, t, (uint32_t)g8, kDomSite | pbits}, J.rk)
                                : philox4x32_10(U4{tile_id, t, (uint32_t)g8, kDomSite | pbits}, J.seed_lo, J.seed_hi);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int g = 2 * g8 + h;
            if (NSEL % 8 != 0 && 4 * g >= NSEL) break;
            const U4 cm = U4{tile_id, t, (uint32_t)g, kDomMask | pbits | (uint32_t)w0};
            const U4 m_lo = RKEYS ? philox4x32_10(cm, J.rk) : philox4x32_10(cm, J.seed_lo, J.seed_hi);
            U4 m_hi = m_lo;
            if (NWT >= 2) {
                const U4 ch = U4{tile_id, t, (uint32_t)g, kDomMask | pbits | (uint32_t)(w0 + 1)};
                m_hi = RKEYS ? philox4x32_10(ch, J.rk) : philox4x32_10(ch, J.seed_lo, J.seed_hi);
            }
            // 128-lane words: the mask blocks of words w0 + 2 and w0 + 3 too
            U4 m_2 = m_lo, m_3 = m_lo;
            if constexpr (NWT == 4) {
                const U4 c2 = U4{tile_id, t, (uint32_t)g, kDomMask | pbits | (uint32_t)(w0 + 2)};
                const U4 c3 = U4{tile_id, t, (uint32_t)g, kDomMask | pbits | (uint32_t)(w0 + 3)};
                m_2 = RKEYS ? philox4x32_10(c2, J.rk) : philox4x32_10(c2, J.seed_lo, J.seed_hi);
                m_3 = RKEYS ? philox4x32_10(c3, J.rk) : philox4x32_10(c3, J.seed_lo, J.seed_hi);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int i8 = 4 * h + r;  // selection index within the block of eight
                if (NSEL % 4 != 0 && 8 * g8 + i8 >= NSEL) break;
                const uint32_t word = pick_word(site_r, i8 >> 1);
                const uint32_t half = (i8 & 1) ? (word >> 16) : (word & 0xFFFFu);
                const uint32_t k = (half * (uint32_t)A) >> 16;
                const int kx = (int)(k % (uint32_t)SX), ky = (int)(k / (uint32_t)SX);
                const int s = (ky + 1) * WW + kx + 1;
                WT* base = sm + ((size_t)s * nthr + tid) * B;
                const size_t rs = (size_t)nthr * B;  // one slot
                if (!RSOS_CHECK_SHARED(J, base - WW * rs, sizeof(WT) * B) ||
                    !RSOS_CHECK_SHARED(J, base + WW * rs, sizeof(WT) * B))
                    continue;
                WT x[B], e[B], w[B], n[B], so[B];
                load_rec<B, WT>(base, x);
                load_rec<B, WT>(base + rs, e);
                load_rec<B, WT>(base - rs, w);
                load_rec<B, WT>(base - WW * rs, n);
                load_rec<B, WT>(base + WW * rs, so);
                WT mk;
                if constexpr (NWT == 4)
                    mk = Word128((unsigned long long)pick_word(m_lo, r) | ((unsigned long long)pick_word(m_hi, r) << 32),
                                 (unsigned long long)pick_word(m_2, r) | ((unsigned long long)pick_word(m_3, r) << 32));
                else
                    mk = mask_word<WT>(m_lo, m_hi, r);
                const WT acc = accept_mask<N, B, WT>(mk, x, e, w, n, so);
                masked_increment<B, WT>(x, acc);
                store_rec<B, WT>(base, x);
                if (HAS00 && (int)k == k00) record_origin_deposits<WT>(J.h00, w0 * 32, acc);
            }
        }
    }

}

// One activation of one sub-tile for one lane-word group (section II):
// stage sub-tile + halo into the thread's private shared-memory slots, run the
// 2a selections in order, write the interior back.
//   sm        block shared-memory base, nthr threads, this thread = tid
//   wp        lane-word group: words wp*NWT .. wp*NWT+NWT-1
//   t, p, q   sweep index, phase, active sub-tile set q = perm[p]
// ASYNC = true stages the window with asynchronous copies (persistent
// engines); otherwise with plain loads through registers.
template <int N, typename WT, int SX, bool HAS00, bool ASYNC = false, int NTHR = 0, bool RKEYS = true>
__device__ __forceinline__ void activate_subtile(const JobDev& J, WT* __restrict__ sm, int tid, int nthr_rt,
                                                 int tx, int ty, int wp, uint32_t t, int p, int q, int ox,
                                                 int oy, int k00)
{
    // A compile-time block size turns every slot offset into an immediate.
    const int nthr = NTHR > 0 ? NTHR : nthr_rt;
    constexpr int B = bits_for_step(N);
    constexpr int SY = SX;
    constexpr int WW = SX + 2;
    constexpr int NWT = (int)(sizeof(WT) / 4);
    const int qx = q & 1, qy = q >> 1;
    const int w0 = wp * NWT;
    const bool whole_record = NWT == J.NW;

    WindowIndex<SX> wi;
    window_index<SX>(J, tx, ty, qx, qy, ox, oy, w0, wi);
    constexpr int UNROLL_ROWS = SX <= 4 ? SY + 2 : 1;

#pragma unroll UNROLL_ROWS
    for (int jj = 0; jj < SY + 2; ++jj) {
#pragma unroll
        for (int ii = 0; ii < SX + 2; ++ii) {
            const bool corner = (jj == 0 || jj == SY + 1) && (ii == 0 || ii == SX + 1);
            if (corner) continue;
            const int s = jj * WW + ii;
            WT* slot = sm + ((size_t)s * nthr + tid) * B;
            const uint32_t* src = J.planes + wi.row[jj] + wi.col[ii];
            if (!RSOS_CHECK_GLOBAL(J, src, (size_t)(B - 1) * J.NW + NWT) || !RSOS_CHECK_SHARED(J, slot, sizeof(WT) * B))
                continue;
            if (ASYNC) {
                stage_record_async<WT, B>(slot, src, J.NW, whole_record);
            } else {
#pragma unroll
                for (int b = 0; b < B; ++b) slot[b] = load_word<WT>(src + (size_t)b * J.NW);
            }
        }
    }
    if (ASYNC) stage_wait_all();

    select_subtile<N, WT, SX, HAS00, NTHR, RKEYS>(J, sm, tid, nthr, (uint32_t)(ty * J.nT + tx), t, p, w0, k00);

    // Recomputed rather than kept live across the selection loop (registers).
    window_index<SX>(J, tx, ty, qx, qy, ox, oy, w0, wi);
#pragma unroll UNROLL_ROWS
    for (int jj = 1; jj <= SY; ++jj) {
#pragma unroll
        for (int ii = 1; ii <= SX; ++ii) {
            const int s = jj * WW + ii;
            const WT* slot = sm + ((size_t)s * nthr + tid) * B;
            uint32_t* dst = J.planes + wi.row[jj] + wi.col[ii];
            if (!RSOS_CHECK_GLOBAL(J, dst, (size_t)(B - 1) * J.NW + NWT) || !RSOS_CHECK_SHARED(J, slot, sizeof(WT) * B))
                continue;
            if (B * sizeof(WT) == 16 && whole_record) {
                store_record16<B, WT>(dst, slot);
            } else {
#pragma unroll
                for (int b = 0; b < B; ++b) *reinterpret_cast<WT*>(dst + (size_t)b * J.NW) = slot[b];
            }
        }
    }
}

// Plain path (one surface, absolute int32 heights, lane 0 of the stream).
template <int SX>
__device__ __forceinline__ void activate_subtile_plain(const JobDev& J, int32_t* __restrict__ sm, int tid,
                                                       int nthr, int tx, int ty, uint32_t t, int p, int q,
                                                       int ox, int oy)
{
    constexpr int SY = SX;
    constexpr int A = SX * SY;
    constexpr int NSEL = 2 * A;
    constexpr int WW = SX + 2;
    const int qx = q & 1, qy = q >> 1;
    const int L = J.L, T = J.T;
    int xs[SX + 2], ys[SY + 2];
#pragma unroll
    for (int ii = 0; ii < SX + 2; ++ii) {
        int x = ox + tx * T + qx * SX + ii - 1;
        xs[ii] = x < 0 ? x + L : (x >= L ? x - L : x);
    }
#pragma unroll
    for (int jj = 0; jj < SY + 2; ++jj) {
        int y = oy + ty * T + qy * SY + jj - 1;
        ys[jj] = y < 0 ? y + L : (y >= L ? y - L : y);
    }
#pragma unroll
    for (int jj = 0; jj < SY + 2; ++jj) {
#pragma unroll
        for (int ii = 0; ii < SX + 2; ++ii) {
            const bool corner = (jj == 0 || jj == SY + 1) && (ii == 0 || ii == SX + 1);
            if (corner) continue;
            sm[(size_t)(jj * WW + ii) * nthr + tid] = J.heights[(size_t)ys[jj] * L + xs[ii]];
        }
    }
    const uint32_t tile_id = (uint32_t)(ty * J.nT + tx);
    const uint32_t pbits = (uint32_t)p << 28;
    U4 site_r = {0u, 0u, 0u, 0u};
#pragma unroll 1
    for (int g = 0; g < (NSEL + 3) / 4; ++g) {
        if ((g & 1) == 0) {
            site_r = philox4x32_10(U4{tile_id, t, (uint32_t)(g >> 1), kDomSite | pbits}, J.seed_lo, J.seed_hi);
        }
        const U4 m = philox4x32_10(U4{tile_id, t, (uint32_t)g, kDomMask | pbits}, J.seed_lo, J.seed_hi);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = 4 * g + r;
            if (NSEL % 4 != 0 && i >= NSEL) break;
            const uint32_t word = pick_word(site_r, ((i >> 1) & 3));
            const uint32_t half = (i & 1) ? (word >> 16) : (word & 0xFFFFu);
            const uint32_t k = (half * (uint32_t)A) >> 16;
            if (!(pick_word(m, r) & 1u)) continue;
            const int s = ((int)(k / (uint32_t)SX) + 1) * WW + (int)(k % (uint32_t)SX) + 1;
            int32_t* base = sm + (size_t)s * nthr + tid;
            const int32_t hx = base[0];
            const int32_t lim = hx - J.N;  // reject if a neighbour sits N below
            const bool ok = base[nthr] != lim && base[-(ptrdiff_t)nthr] != lim &&
                            base[-(ptrdiff_t)WW * nthr] != lim && base[(size_t)WW * nthr] != lim;
            if (ok) base[0] = hx + 1;
        }
    }
#pragma unroll
    for (int jj = 1; jj <= SY; ++jj) {
#pragma unroll
        for (int ii = 1; ii <= SX; ++ii) {
            J.heights[(size_t)ys[jj] * L + xs[ii]] = sm[(size_t)(jj * WW + ii) * nthr + tid];
        }
    }
}

#endif  // __CUDACC__

}  // namespace rsos

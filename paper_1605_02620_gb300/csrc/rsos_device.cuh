// Device-side data structures and the sub-tile activation of the RSOS
// double-tiling sweep (section II of the paper; Eq. 6 for the update rule).
//
// Data layout in HBM (multisurface path).  A job of S surfaces has
// NW = ceil(S/32) lane words; bit j of word w is surface 32*w + j.  The
// residue h mod 2^B of every site is stored in B bit planes.  Within a plane
// the sites are ordered  [y][x mod T][x div T][w]  ("class-interleaved" by the
// tile edge T): the same column class of consecutive tiles is contiguous, so a
// warp whose threads work on consecutive tiles reads and writes one contiguous
// run of words whatever the random tiling origin of the sweep is.
//
// Shared memory (per thread, private): the active sub-tile plus its one-site
// halo, (SX+2) x (SY+2) slots (corners unused), each slot B words of the
// thread's lane-word group, stored [slot][plane][thread] so that every thread
// owns its own bank column: random per-thread site choices never conflict.
#pragma once
#include "philox.cuh"
#include "rsos_logic.cuh"

namespace rsos {

struct JobDev {
    uint32_t* planes;   // multisurface: B planes of L*L*NW words
    int32_t* heights;   // plain path: L*L int32, row-major
    int64_t* h00;       // absolute height of site (0,0) per lane (NW*32)
    int32_t L, T, nT;   // lattice edge, tile edge (square tiles), tiles per row
    int32_t NW;         // 32-lane words per site and plane
    int32_t NWP;        // thread groups per tile (NW / words per thread)
    int32_t N, B;
    int32_t phase_order;
    uint32_t seed_lo, seed_hi;
    RoundKeys rk;       // Philox round keys of the seed
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

#if defined(__CUDACC__)

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

// Global loads of lattice words.  CG = true bypasses L1 (ld.global.cg): in the
// persistent engine another block may have rewritten the line since this SM
// last cached it.
template <typename WT, bool CG>
__device__ __forceinline__ WT load_word(const uint32_t* p)
{
    if (CG) {
        if (sizeof(WT) == 8) return (WT)__ldcg(reinterpret_cast<const unsigned long long*>(p));
        return (WT)__ldcg(reinterpret_cast<const unsigned int*>(p));
    }
    return *reinterpret_cast<const WT*>(p);
}

// Word offsets of the window columns i = -1..SX and rows j = -1..SY of the
// active sub-tile of tile (tx, ty) in the sweep's tiling.
template <int SX>
struct WindowIndex {
    size_t col[SX + 2];
    size_t row[SX + 2];
};

template <int SX>
__device__ __forceinline__ void window_index(const JobDev& J, int tx, int ty, int qx, int qy, int ox,
                                             int oy, int w0, WindowIndex<SX>& wi)
{
    constexpr int T = 2 * SX;  // square tiles: the tile edge is known at compile time
    const int nT = J.nT, L = J.L;
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
        wi.col[ii] = ((size_t)xr * nT + col) * J.NW + w0;
    }
#pragma unroll
    for (int jj = 0; jj < SX + 2; ++jj) {
        int y = oy + ty * T + qy * SX + jj - 1;  // in [-1, L + T)
        y = y < 0 ? y + L : (y >= L ? y - L : y);
        wi.row[jj] = (size_t)y * ((size_t)T * nT * J.NW);
    }
}

// One activation of one sub-tile for one lane-word group (section II):
// stage sub-tile + halo into the thread's private shared-memory slots, run the
// 2a selections in order, write the interior back.
//   sm        block shared-memory base, nthr threads, this thread = tid
//   wp        lane-word group: words wp*NWT .. wp*NWT+NWT-1
//   t, p, q   sweep index, phase, active sub-tile set q = perm[p]
template <int N, typename WT, int SX, bool HAS00, bool CG = false, int NTHR = 0, bool RKEYS = true>
__device__ __forceinline__ void activate_subtile(const JobDev& J, WT* __restrict__ sm, int tid, int nthr_rt,
                                                 int tx, int ty, int wp, uint32_t t, int p, int q, int ox,
                                                 int oy, int k00)
{
    // A compile-time block size turns every slot offset into an immediate.
    const int nthr = NTHR > 0 ? NTHR : nthr_rt;
    constexpr int B = bits_for_step(N);
    constexpr int SY = SX;
    constexpr int A = SX * SY;
    constexpr int NSEL = 2 * A;
    constexpr int WW = SX + 2;
    constexpr int NWT = (int)(sizeof(WT) / 4);
    const int qx = q & 1, qy = q >> 1;
    const int w0 = wp * NWT;
    const size_t plane = (size_t)J.L * J.L * J.NW;

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
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const WT v = load_word<WT, CG>(J.planes + b * plane + wi.row[jj] + wi.col[ii]);
                sm[(size_t)(s * B + b) * nthr + tid] = v;
            }
        }
    }

    const uint32_t tile_id = (uint32_t)(ty * J.nT + tx);
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
            if (NWT == 2) {
                const U4 ch = U4{tile_id, t, (uint32_t)g, kDomMask | pbits | (uint32_t)(w0 + 1)};
                m_hi = RKEYS ? philox4x32_10(ch, J.rk) : philox4x32_10(ch, J.seed_lo, J.seed_hi);
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
                WT* base = sm + (size_t)s * B * nthr + tid;
                WT x[B], e[B], w[B], n[B], so[B];
#pragma unroll
                for (int b = 0; b < B; ++b) {
                    x[b] = base[(size_t)b * nthr];
                    e[b] = base[(size_t)(B + b) * nthr];
                    w[b] = base[-(ptrdiff_t)(B - b) * nthr];
                    n[b] = base[-(ptrdiff_t)(WW * B - b) * nthr];
                    so[b] = base[(size_t)(WW * B + b) * nthr];
                }
                const WT acc = accept_mask<N, B, WT>(mask_word<WT>(m_lo, m_hi, r), x, e, w, n, so);
                masked_increment<B, WT>(x, acc);
#pragma unroll
                for (int b = 0; b < B; ++b) base[(size_t)b * nthr] = x[b];
                if (HAS00 && (int)k == k00) record_origin_deposits<WT>(J.h00, w0 * 32, acc);
            }
        }
    }

    // Recomputed rather than kept live across the selection loop (registers).
    window_index<SX>(J, tx, ty, qx, qy, ox, oy, w0, wi);
#pragma unroll UNROLL_ROWS
    for (int jj = 1; jj <= SY; ++jj) {
#pragma unroll
        for (int ii = 1; ii <= SX; ++ii) {
            const int s = jj * WW + ii;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                *reinterpret_cast<WT*>(J.planes + b * plane + wi.row[jj] + wi.col[ii]) =
                    sm[(size_t)(s * B + b) * nthr + tid];
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

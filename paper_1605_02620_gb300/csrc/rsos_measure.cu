// Exact width measurement (Eq. 2) of multisurface-coded lattices, plus the
// flat-start initialisation (section II).
//
// The coded lattice holds h mod 2^B per site and lane.  Neighbour
// differences decode uniquely because |h(x) - h(n)| <= N < 2^(B-1): the B-bit
// residue of h(n) - h(x) read as a two's-complement number IS the difference.
// Heights relative to site (0,0) follow by summing differences along row 0
// and then down every column; with the tracked absolute height h00 of site
// (0,0) per lane,
//     sum h   = L^2 h00 + sum rel
//     sum h^2 = L^2 h00^2 + 2 h00 sum rel + sum rel^2
// in 128-bit integers.  Kernels:
//   row0_prefix_kernel   rel(x, 0) for every lane (one block per lane word)
//   column_walk_kernel   per column and lane, sum rel and sum rel^2 down y,
//                        in row segments combined exactly in order
//   finalize_kernel      per lane, 128-bit totals combined with h00
#include "rsos_launch.h"

namespace rsos {

__device__ __forceinline__ int lane_residue(const JobDev& J, int x, int y, int w, int lane)
{
    const size_t rec = site_record(J, x, y);
    int v = 0;
    for (int b = 0; b < J.B; ++b) v |= (int)((J.planes[plane_word(J, rec, b, w)] >> lane) & 1u) << b;
    return v;
}

// h(b) - h(a) from the residues a, b (B-bit two's complement).
__device__ __forceinline__ int residue_diff(int a, int b, int B)
{
    const int d = (b - a) & ((1 << B) - 1);
    return d >= (1 << (B - 1)) ? d - (1 << B) : d;
}

// rel(x, 0) of every lane of word blockIdx.x, in tiles of 1024 sites: thread
// (lane j, sub-chunk c) sums the differences of 32 consecutive sites, a
// per-lane scan over the 32 sub-chunks gives the offsets, and the running
// carry joins the tiles.
__global__ void __launch_bounds__(1024) row0_prefix_kernel(JobDev J, int32_t* __restrict__ row0)
{
    __shared__ uint32_t words[4][1025];
    __shared__ int32_t chunk_sum[32][33];
    const int w = blockIdx.x, lane = threadIdx.x & 31, c = threadIdx.x >> 5;
    const int L = J.L, B = J.B;
    int32_t* out = row0 + (size_t)(w * 32 + lane) * L;
    int carry = 0;
    for (int X0 = 0; X0 < L; X0 += 1024) {
        __syncthreads();
        for (int k = threadIdx.x; k < 1025; k += blockDim.x) {
            const int x = X0 + k;
            for (int b = 0; b < B; ++b) words[b][k] = x < L ? J.planes[plane_word(J, site_record(J, x, 0), b, w)] : 0u;
        }
        __syncthreads();
        const int i0 = 32 * c;
        int v = 0;
        for (int b = 0; b < B; ++b) v |= (int)((words[b][i0] >> lane) & 1u) << b;
        int loc[32];
        int acc = 0;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            loc[i] = acc;
            const int x = X0 + i0 + i;
            if (x + 1 < L) {
                int vn = 0;
                for (int b = 0; b < B; ++b) vn |= (int)((words[b][i0 + i + 1] >> lane) & 1u) << b;
                acc += residue_diff(v, vn, B);
                v = vn;
            }
        }
        chunk_sum[c][lane] = acc;
        __syncthreads();
        int off = carry, total = carry;
        for (int cc = 0; cc < 32; ++cc) {
            const int sc = chunk_sum[cc][lane];
            if (cc < c) off += sc;
            total += sc;
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const int x = X0 + i0 + i;
            if (x < L) out[x] = off + loc[i];
        }
        carry = total;
    }
}

// Column sums, exact.  Block (lane group blockIdx.x of 8 lanes, column block
// blockIdx.y = 32 columns of one class, word blockIdx.z) with 8 warps; warp s
// walks row segment s of the 32 columns.  Relative to its first row a
// segment yields, per lane, (Delta, sum r, sum r^2); the segments combine in
// order:  offset o accumulates the Deltas and a segment of n rows adds
// n o + sum r  and  n o^2 + 2 o sum r + sum r^2.  Adding rel(x, 0) gives the
// column totals, which a warp reduction sums over the 32 columns.
constexpr int kSeg = 8;

__global__ void __launch_bounds__(256) column_walk_kernel(JobDev J, const int32_t* __restrict__ row0,
                                                          int S_pad, int64_t* __restrict__ partial)
{
    __shared__ int32_t sD[kSeg][8][32];
    __shared__ int32_t sS1[kSeg][8][32];
    __shared__ long long sS2[kSeg][8][32];
    const int lg = blockIdx.x, cb = blockIdx.y, w = blockIdx.z;
    const int T = J.T, nT = J.nT, L = J.L, B = J.B;
    const int u = cb % T;
    const int col = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const int m = (cb / T) * 32 + col;
    const int x = m * T + u;
    const bool valid = m < nT && x < L;  // (+1) tilings: last class columns partly unused
    const int RL = (L + kSeg - 1) / kSeg;
    const int y0 = min(L, seg * RL), y1 = min(L, y0 + RL);
    int r[8], s1[8], vprev[8];
    long long s2[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        r[k] = 0;
        s1[k] = 0;
        s2[k] = 0;
        vprev[k] = 0;
    }
    if (valid && y0 < y1) {
        const size_t row_stride = (size_t)T * nT * B * J.NW;  // words per lattice row
        const uint32_t* base = J.planes + plane_word(J, site_record(J, x, y0), 0, w);
        const int sh = lg * 8;
        // lane k's residue from the plane words of one site (bits sh + k)
        auto residues = [&](const uint32_t (&wv)[4], int (&v)[8]) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                int a = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (b < B) a |= (int)((wv[b] >> (sh + k)) & 1u) << b;
                v[k] = a;
            }
        };
        const int hs = 32 - B;  // B-bit two's complement difference by shifts
        {
            uint32_t wv[4] = {0u, 0u, 0u, 0u};
            for (int b = 0; b < B; ++b) wv[b] = base[(size_t)b * J.NW];
            residues(wv, vprev);
        }
        // Rows y0+1 .. y1-1 contribute to the sums; row y1 (if inside the
        // lattice) only closes the segment's difference.  Eight rows' words
        // are loaded before any is decoded (memory-level parallelism).
        const int ylast = y1 < L ? y1 : L - 1;
        int y = y0 + 1;
        for (; y + 7 <= ylast; y += 8) {
            uint32_t wv[8][4];
#pragma unroll
            for (int u8 = 0; u8 < 8; ++u8)
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    wv[u8][b] = b < B ? __ldg(base + (size_t)(y - y0 + u8) * row_stride + (size_t)b * J.NW) : 0u;
#pragma unroll
            for (int u8 = 0; u8 < 8; ++u8) {
                int v[8];
                residues(wv[u8], v);
                const bool inside = y + u8 < y1;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    r[k] += ((v[k] - vprev[k]) << hs) >> hs;
                    vprev[k] = v[k];
                    if (inside) {
                        s1[k] += r[k];
                        s2[k] += (long long)r[k] * r[k];
                    }
                }
            }
        }
        for (; y <= ylast; ++y) {
            uint32_t wv[4] = {0u, 0u, 0u, 0u};
            for (int b = 0; b < B; ++b) wv[b] = base[(size_t)(y - y0) * row_stride + (size_t)b * J.NW];
            int v[8];
            residues(wv, v);
            const bool inside = y < y1;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                r[k] += ((v[k] - vprev[k]) << hs) >> hs;
                vprev[k] = v[k];
                if (inside) {
                    s1[k] += r[k];
                    s2[k] += (long long)r[k] * r[k];
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        sD[seg][k][col] = r[k];
        sS1[seg][k][col] = s1[k];
        sS2[seg][k][col] = s2[k];
    }
    __syncthreads();
    if (seg != 0) return;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int lane = lg * 8 + k;
        long long t1 = 0, t2 = 0;
        if (valid) {
            long long off = 0;
            for (int sg = 0; sg < kSeg; ++sg) {
                const int a0 = min(L, sg * RL), a1 = min(L, a0 + RL);
                const long long n = a1 - a0;
                if (n <= 0) break;
                const long long sr = sS1[sg][k][col], sr2 = sS2[sg][k][col];
                t1 += n * off + sr;
                t2 += n * off * off + 2 * off * sr + sr2;
                off += sD[sg][k][col];
            }
            const long long rel0 = row0[(size_t)(w * 32 + lane) * L + x];
            t2 += (long long)L * rel0 * rel0 + 2 * rel0 * t1;
            t1 += (long long)L * rel0;
        }
        for (int o = 16; o > 0; o >>= 1) {
            t1 += __shfl_down_sync(0xffffffffu, t1, o);
            t2 += __shfl_down_sync(0xffffffffu, t2, o);
        }
        if (col == 0) {
            const size_t rr = ((size_t)cb * S_pad + (size_t)w * 32 + lane) * 2;
            partial[rr] = t1;
            partial[rr + 1] = t2;
        }
    }
}

// Plain path: absolute heights, one partial row per block (lane 0 only).
__global__ void __launch_bounds__(256) plain_sum_kernel(const int32_t* __restrict__ h, long long n,
                                                        int64_t* __restrict__ partial)
{
    long long a = 0, b = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long v = h[k];
        a += v;
        b += v * v;
    }
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    __shared__ long long sa[8], sb[8];
    if ((threadIdx.x & 31) == 0) {
        sa[threadIdx.x >> 5] = a;
        sb[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long ta = 0, tb = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            ta += sa[k];
            tb += sb[k];
        }
        partial[(size_t)blockIdx.x * 2] = ta;
        partial[(size_t)blockIdx.x * 2 + 1] = tb;
    }
}

// Per lane (one block each): 128-bit totals over the partial rows, then the
// absolute sums with h00.
__global__ void __launch_bounds__(128) finalize_kernel(const int64_t* __restrict__ partial, int nrows, int S_pad,
                                                       int L, const int64_t* __restrict__ h00,
                                                       int64_t* __restrict__ rec, int rec_stride)
{
    __shared__ __int128 a1[128], a2[128];
    const int lane = blockIdx.x;
    __int128 s1 = 0, s2 = 0;
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
        s1 += (__int128)partial[((size_t)r * S_pad + lane) * 2];
        s2 += (__int128)partial[((size_t)r * S_pad + lane) * 2 + 1];
    }
    a1[threadIdx.x] = s1;
    a2[threadIdx.x] = s2;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            a1[threadIdx.x] += a1[threadIdx.x + o];
            a2[threadIdx.x] += a2[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    s1 = a1[0];
    s2 = a2[0];
    const __int128 h0 = h00 ? (__int128)h00[lane] : (__int128)0;
    const __int128 area = (__int128)L * L;
    const __int128 sh = area * h0 + s1;
    const __int128 sh2 = area * h0 * h0 + 2 * h0 * s1 + s2;
    rec[(size_t)lane * rec_stride + 0] = (int64_t)(uint64_t)sh;
    rec[(size_t)lane * rec_stride + 1] = (int64_t)(sh >> 64);
    rec[(size_t)lane * rec_stride + 2] = (int64_t)(uint64_t)sh2;
    rec[(size_t)lane * rec_stride + 3] = (int64_t)(sh2 >> 64);
}

// ---- Third and fourth power sums (height-distribution skewness and
// kurtosis, section III.C).  Same walk as column_walk_kernel, also carrying
// sum r^3 (int64: |r| <= L/8 * N in a segment) and sum r^4 (128-bit); the
// segments and the row-0 offsets combine by binomial expansion in 128 bits.
__device__ __forceinline__ __int128 shfl_down_i128(__int128 v, int o)
{
    const unsigned long long lo = __shfl_down_sync(0xffffffffu, (unsigned long long)v, o);
    const long long hi = __shfl_down_sync(0xffffffffu, (long long)(v >> 64), o);
    return (__int128)(((unsigned __int128)(unsigned long long)hi << 64) | lo);
}

// Per (column block, lane): sum over the block's columns of rel^k, k = 1..4,
// into partial[(cb * S_pad + lane) * 6 + ...] = t1, t2, t3 lo, t3 hi, t4 lo, t4 hi.
__global__ void __launch_bounds__(256) column_moments_kernel(JobDev J, const int32_t* __restrict__ row0, int S_pad,
                                                             int64_t* __restrict__ partial)
{
    extern __shared__ __align__(16) unsigned char msm[];
    // [kSeg][8][32] each: D, S1 (int32), S2, S3 (int64), S4 (int128)
    int32_t* sD = reinterpret_cast<int32_t*>(msm);
    int32_t* sS1 = sD + kSeg * 8 * 32;
    long long* sS2 = reinterpret_cast<long long*>(sS1 + kSeg * 8 * 32);
    long long* sS3 = sS2 + kSeg * 8 * 32;
    __int128* sS4 = reinterpret_cast<__int128*>(sS3 + kSeg * 8 * 32);
    const int lg = blockIdx.x, cb = blockIdx.y, w = blockIdx.z;
    const int T = J.T, nT = J.nT, L = J.L, B = J.B;
    const int u = cb % T;
    const int col = threadIdx.x & 31, seg = threadIdx.x >> 5;
    const int m = (cb / T) * 32 + col;
    const int x = m * T + u;
    const bool valid = m < nT && x < L;  // (+1) tilings: last class columns partly unused
    const int RL = (L + kSeg - 1) / kSeg;
    const int y0 = min(L, seg * RL), y1 = min(L, y0 + RL);
    int r[8], s1[8], vprev[8];
    long long s2[8], s3[8];
    __int128 s4[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        r[k] = 0;
        s1[k] = 0;
        s2[k] = 0;
        s3[k] = 0;
        s4[k] = 0;
        vprev[k] = 0;
    }
    if (valid && y0 < y1) {
        const size_t row_stride = (size_t)T * nT * B * J.NW;
        const uint32_t* base = J.planes + plane_word(J, site_record(J, x, y0), 0, w);
        const int sh = lg * 8, hs = 32 - B;
        auto residues = [&](const uint32_t* wv, int* v) {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                int a = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (b < B) a |= (int)((wv[b] >> (sh + k)) & 1u) << b;
                v[k] = a;
            }
        };
        {
            uint32_t wv[4] = {0u, 0u, 0u, 0u};
            for (int b = 0; b < B; ++b) wv[b] = base[(size_t)b * J.NW];
            residues(wv, vprev);
        }
        const int ylast = y1 < L ? y1 : L - 1;
        for (int y = y0 + 1; y <= ylast; ++y) {
            uint32_t wv[4] = {0u, 0u, 0u, 0u};
            for (int b = 0; b < B; ++b) wv[b] = __ldg(base + (size_t)(y - y0) * row_stride + (size_t)b * J.NW);
            int v[8];
            residues(wv, v);
            const bool inside = y < y1;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                r[k] += ((v[k] - vprev[k]) << hs) >> hs;
                vprev[k] = v[k];
                if (inside) {
                    const long long rr = (long long)r[k] * r[k];
                    s1[k] += r[k];
                    s2[k] += rr;
                    s3[k] += rr * r[k];
                    s4[k] += (__int128)(rr * rr);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int i = (seg * 8 + k) * 32 + col;
        sD[i] = r[k];
        sS1[i] = s1[k];
        sS2[i] = s2[k];
        sS3[i] = s3[k];
        sS4[i] = s4[k];
    }
    __syncthreads();
    if (seg != 0) return;
#pragma unroll 1
    for (int k = 0; k < 8; ++k) {
        const int lane = lg * 8 + k;
        __int128 t1 = 0, t2 = 0, t3 = 0, t4 = 0;
        if (valid) {
            // segments in order: a segment of n rows at offset o adds
            // sum (o + r)^j, expanded binomially
            __int128 off = 0;
            for (int sg = 0; sg < kSeg; ++sg) {
                const int a0 = min(L, sg * RL), a1 = min(L, a0 + RL);
                const __int128 n = a1 - a0;
                if (n <= 0) break;
                const int i = (sg * 8 + k) * 32 + col;
                const __int128 q1 = sS1[i], q2 = sS2[i], q3 = sS3[i], q4 = sS4[i];
                const __int128 o2 = off * off, o3 = o2 * off;
                t1 += n * off + q1;
                t2 += n * o2 + 2 * off * q1 + q2;
                t3 += n * o3 + 3 * o2 * q1 + 3 * off * q2 + q3;
                t4 += n * o3 * off + 4 * o3 * q1 + 6 * o2 * q2 + 4 * off * q3 + q4;
                off += sD[i];
            }
            // shift the column by its row-0 value rel(x, 0)
            const __int128 c = row0[(size_t)(w * 32 + lane) * L + x];
            const __int128 c2 = c * c, c3 = c2 * c, nL = L;
            t4 += nL * c3 * c + 4 * c3 * t1 + 6 * c2 * t2 + 4 * c * t3;
            t3 += nL * c3 + 3 * c2 * t1 + 3 * c * t2;
            t2 += nL * c2 + 2 * c * t1;
            t1 += nL * c;
        }
        for (int o = 16; o > 0; o >>= 1) {
            t1 += shfl_down_i128(t1, o);
            t2 += shfl_down_i128(t2, o);
            t3 += shfl_down_i128(t3, o);
            t4 += shfl_down_i128(t4, o);
        }
        if (col == 0) {
            int64_t* out = partial + ((size_t)cb * S_pad + (size_t)w * 32 + lane) * 6;
            out[0] = (int64_t)t1;  // |t1|, |t2| of 32 columns fit 64 bits
            out[1] = (int64_t)t2;
            out[2] = (int64_t)(uint64_t)t3;
            out[3] = (int64_t)(t3 >> 64);
            out[4] = (int64_t)(uint64_t)t4;
            out[5] = (int64_t)(t4 >> 64);
        }
    }
}

constexpr size_t kMomentsSmem = (size_t)kSeg * 8 * 32 * (4 + 4 + 8 + 8 + 16);

// Plain path: power sums of the int32 heights, six words per block.
__global__ void __launch_bounds__(256) plain_moments_kernel(const int32_t* __restrict__ h, long long n,
                                                            int64_t* __restrict__ partial)
{
    __int128 a[4] = {0, 0, 0, 0};
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const __int128 v = h[k], v2 = v * v;
        a[0] += v;
        a[1] += v2;
        a[2] += v2 * v;
        a[3] += v2 * v2;
    }
    __shared__ __int128 sa[4][256];
#pragma unroll
    for (int j = 0; j < 4; ++j) sa[j][threadIdx.x] = a[j];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
#pragma unroll
            for (int j = 0; j < 4; ++j) sa[j][threadIdx.x] += sa[j][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int64_t* out = partial + (size_t)blockIdx.x * 6;
        out[0] = (int64_t)sa[0][0];
        out[1] = (int64_t)sa[1][0];
        out[2] = (int64_t)(uint64_t)sa[2][0];
        out[3] = (int64_t)(sa[2][0] >> 64);
        out[4] = (int64_t)(uint64_t)sa[3][0];
        out[5] = (int64_t)(sa[3][0] >> 64);
    }
}

// Per lane: 128-bit totals of sum rel^k over the partial rows, then
// sum h^k = sum_j C(k, j) h00^(k-j) sum rel^j  (sum rel^0 = L^2), into
// rec[lane * 8 ...] = sum h, sum h^2, sum h^3, sum h^4 as (lo, hi) pairs.
__global__ void __launch_bounds__(128) finalize_moments_kernel(const int64_t* __restrict__ partial, int nrows,
                                                               int S_pad, int L, const int64_t* __restrict__ h00,
                                                               int64_t* __restrict__ rec)
{
    __shared__ __int128 acc[4][128];
    const int lane = blockIdx.x;
    __int128 s[4] = {0, 0, 0, 0};
    for (int r = threadIdx.x; r < nrows; r += blockDim.x) {
        const int64_t* p = partial + ((size_t)r * S_pad + lane) * 6;
        s[0] += (__int128)p[0];
        s[1] += (__int128)p[1];
        s[2] += (__int128)(((unsigned __int128)(uint64_t)p[3] << 64) | (uint64_t)p[2]);
        s[3] += (__int128)(((unsigned __int128)(uint64_t)p[5] << 64) | (uint64_t)p[4]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j][threadIdx.x] = s[j];
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j][threadIdx.x] += acc[j][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const __int128 a = h00 ? (__int128)h00[lane] : (__int128)0;
    const __int128 n = (__int128)L * L, q1 = acc[0][0], q2 = acc[1][0], q3 = acc[2][0], q4 = acc[3][0];
    const __int128 a2 = a * a, a3 = a2 * a;
    const __int128 out[4] = {n * a + q1, n * a2 + 2 * a * q1 + q2, n * a3 + 3 * a2 * q1 + 3 * a * q2 + q3,
                             n * a3 * a + 4 * a3 * q1 + 6 * a2 * q2 + 4 * a * q3 + q4};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        rec[(size_t)lane * 8 + 2 * j] = (int64_t)(uint64_t)out[j];
        rec[(size_t)lane * 8 + 2 * j + 1] = (int64_t)(out[j] >> 64);
    }
}

// Heights of one lane: thread per column, walking down y from row 0.
__global__ void heights_kernel(JobDev J, int lane, const int32_t* __restrict__ row0, int64_t* __restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= J.L) return;
    const int w = lane >> 5, bit = lane & 31;
    const int64_t h0 = J.h00[lane];
    int rel = row0[(size_t)lane * J.L + x];
    int vprev = lane_residue(J, x, 0, w, bit);
    out[x] = h0 + rel;
    for (int y = 1; y < J.L; ++y) {
        const int v = lane_residue(J, x, y, w, bit);
        rel += residue_diff(vprev, v, J.B);
        vprev = v;
        out[(size_t)y * J.L + x] = h0 + rel;
    }
}

__global__ void plain_heights_kernel(const int32_t* __restrict__ h, long long n, int64_t* __restrict__ out)
{
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        out[k] = h[k];
}

__global__ void zero_kernel(uint4* __restrict__ p, size_t n16, unsigned char* __restrict__ tail, size_t ntail)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n16; k += stride) p[k] = make_uint4(0, 0, 0, 0);
    if (blockIdx.x == 0 && threadIdx.x < ntail) tail[threadIdx.x] = 0;
}

int measure_blocks(const JobDev& J, bool plain)
{
    if (plain) return 256;
    return J.T * ((J.nT + 31) / 32);
}

cudaError_t launch_measure(const JobDev& J, bool plain, int S_pad, int32_t* row0, int64_t* partial, int ncb_capacity,
                           int64_t* rec, int rec_stride, cudaStream_t s)
{
    const int ncb = measure_blocks(J, plain);
    if (ncb > ncb_capacity) return cudaErrorInvalidValue;
    if (plain) {
        plain_sum_kernel<<<ncb, 256, 0, s>>>(J.heights, (long long)J.L * J.L, partial);
        finalize_kernel<<<1, 128, 0, s>>>(partial, ncb, 1, J.L, nullptr, rec, rec_stride);
        return cudaGetLastError();
    }
    row0_prefix_kernel<<<J.NW, 1024, 0, s>>>(J, row0);
    column_walk_kernel<<<dim3(4, ncb, J.NW), 256, 0, s>>>(J, row0, S_pad, partial);
    finalize_kernel<<<S_pad, 128, 0, s>>>(partial, ncb, S_pad, J.L, J.h00, rec, rec_stride);
    return cudaGetLastError();
}

cudaError_t launch_moments(const JobDev& J, bool plain, int S_pad, int32_t* row0, int64_t* partial,
                           int ncb_capacity, int64_t* rec8, cudaStream_t s)
{
    const int ncb = measure_blocks(J, plain);
    if (ncb > ncb_capacity) return cudaErrorInvalidValue;
    if (plain) {
        plain_moments_kernel<<<ncb, 256, 0, s>>>(J.heights, (long long)J.L * J.L, partial);
        finalize_moments_kernel<<<1, 128, 0, s>>>(partial, ncb, 1, J.L, nullptr, rec8);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(column_moments_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMomentsSmem);
    if (e != cudaSuccess) return e;
    row0_prefix_kernel<<<J.NW, 1024, 0, s>>>(J, row0);
    column_moments_kernel<<<dim3(4, ncb, J.NW), 256, kMomentsSmem, s>>>(J, row0, S_pad, partial);
    finalize_moments_kernel<<<S_pad, 128, 0, s>>>(partial, ncb, S_pad, J.L, J.h00, rec8);
    return cudaGetLastError();
}

cudaError_t launch_heights(const JobDev& J, bool plain, int lane, int32_t* row0, int64_t* out, cudaStream_t s)
{
    if (plain) {
        plain_heights_kernel<<<256, 256, 0, s>>>(J.heights, (long long)J.L * J.L, out);
        return cudaGetLastError();
    }
    row0_prefix_kernel<<<J.NW, 1024, 0, s>>>(J, row0);
    heights_kernel<<<(J.L + 127) / 128, 128, 0, s>>>(J, lane, row0, out);
    return cudaGetLastError();
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s)
{
    const size_t n16 = bytes / 16, ntail = bytes % 16;
    size_t blocks = (n16 + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks == 0) blocks = 1;
    zero_kernel<<<(unsigned)blocks, 256, 0, s>>>(reinterpret_cast<uint4*>(p), n16,
                                                  reinterpret_cast<unsigned char*>(p) + n16 * 16, ntail);
    return cudaGetLastError();
}

}  // namespace rsos

// Geometry of the (+1) tilings of the decomposition check (section III.C:
// domains of 6(+1) x 10(+1) sites).  Host and device.
//
// Along an axis of L sites and base edge T there are n = L div T tiles; the
// first r = L mod T of them are one site wider, so the widths add up to L
// (r <= n).  In pattern coordinates tile c starts at c T + min(c, r).  Every
// tile is halved into floor(w/2) sites (half 0) and the rest (half 1); the
// halves of one set are always separated by a half of the other set, so a set
// can be updated in parallel (section II).  The pattern repeats after T sites
// when T divides L, else after L: the per-sweep origin is uniform over that
// period.  With T even and dividing L this is the regular tiling.
//
// Lattice layout for these tilings: the regular tiling's, site records
// interleaved by column class of the x base edge T, record index
// (y T + x mod T) nT + x div T, with nT = ceil(L / T) class columns per row
// (when T does not divide L the last class columns of a row stay unused).
// Tiles of base width are T apart, so for one window slot the records of
// consecutive tiles are consecutive and a warp's access is one contiguous
// run; the measurement kernels read this layout unchanged.
#pragma once
#include "rsos_common.cuh"

namespace rsos {

struct GenAxis {
    int32_t T, n, r;
};

RSOS_HD GenAxis gen_axis(int L, int T)
{
    return GenAxis{T, L / T, L % T};
}

RSOS_HD bool gen_axis_valid(int L, int T)
{
    return T >= 2 && L >= T && L % T <= L / T;
}

RSOS_HD int gen_period(int L, int T)
{
    return L % T == 0 ? T : L;
}

// Start (pattern coordinate) and width of half `half` of tile c.
RSOS_HD void gen_half(const GenAxis& a, int c, int half, int& start, int& width)
{
    const int X = c * a.T + (c < a.r ? c : a.r);
    const int w = a.T + (c < a.r ? 1 : 0);
    const int w0 = w >> 1;
    start = X + (half ? w0 : 0);
    width = half ? w - w0 : w0;
}

// Tile holding pattern coordinate u in [0, L).
RSOS_HD int gen_tile_of(const GenAxis& a, int u)
{
    const int wide = a.r * (a.T + 1);
    return u < wide ? u / (a.T + 1) : a.r + (u - wide) / a.T;
}

// Widest half of the axis (the window of a sub-tile is this plus a halo).
RSOS_HD int gen_max_half(const GenAxis& a)
{
    return (a.T + (a.r > 0 ? 1 : 0) + 1) >> 1;
}

// v in [-L, 2L) -> v mod L.
RSOS_HD int gen_wrap(int v, int L)
{
    return v < 0 ? v + L : (v >= L ? v - L : v);
}

// Class columns of a row: ceil(L / T).
RSOS_HD int gen_classes(int L, int T)
{
    return (L + T - 1) / T;
}

// Column x of the lattice with its class coordinates (x = q T + r).  The
// window loops walk columns with gen_col_next instead of dividing per slot.
struct GenCol {
    int32_t x, q, r;
};

// Column of (unwrapped) coordinate v in [-L, 2L).
RSOS_HD GenCol gen_col(int L, int T, int v)
{
    const int x = gen_wrap(v, L);
    const int q = x / T;
    return GenCol{x, q, x - q * T};
}

// The next column to the east (periodic).
RSOS_HD void gen_col_next(GenCol& c, int L, int T)
{
    if (++c.x == L) {
        c = GenCol{0, 0, 0};
        return;
    }
    if (++c.r == T) {
        c.r = 0;
        ++c.q;
    }
}

// Word offset of column c within a row of records (rec_words words each).
RSOS_HD size_t gen_col_words(const GenCol& c, int nT, size_t rec_words)
{
    return ((size_t)c.r * (size_t)nT + (size_t)c.q) * rec_words;
}

// Word offset of the row of (unwrapped) coordinate v in [-L, 2L).
RSOS_HD size_t gen_row_words(int L, int T, int nT, size_t rec_words, int v)
{
    return (size_t)gen_wrap(v, L) * (size_t)T * (size_t)nT * rec_words;
}

// floor(k / w) for k < 4096 and 1 <= w <= 16 by a multiply with
// inv = ceil(2^16 / w): k inv / 2^16 exceeds k / w by k e / (w 2^16) with
// e = inv w - 2^16 < w, which stays below 1 / w (the distance from k / w to
// the next integer) while k e < 2^16.
RSOS_HD uint32_t gen_inv(uint32_t w)
{
    return (65536u + w - 1u) / w;
}

RSOS_HD uint32_t gen_div(uint32_t k, uint32_t inv)
{
    return (k * inv) >> 16;
}

struct GenTiling {
    GenAxis x, y;
    int32_t max_w, max_h;  // widest half along x and y
};

RSOS_HD GenTiling gen_tiling(int L, int Tx, int Ty)
{
    GenTiling G;
    G.x = gen_axis(L, Tx);
    G.y = gen_axis(L, Ty);
    G.max_w = gen_max_half(G.x);
    G.max_h = gen_max_half(G.y);
    return G;
}

// Where site (0,0) lies in the tiling of one sweep (origin ox, oy).
struct GenOrigin {
    int tx, ty;  // tile
    int q;       // sub-tile set
    int k;       // site index inside the sub-tile (row-major, k = ky w + kx)
};

RSOS_HD GenOrigin gen_locate_origin_site(int L, const GenTiling& G, int ox, int oy)
{
    const int u = ox == 0 ? 0 : L - ox, v = oy == 0 ? 0 : L - oy;
    GenOrigin o;
    o.tx = gen_tile_of(G.x, u);
    o.ty = gen_tile_of(G.y, v);
    int s0, w0, s1, w1;
    gen_half(G.x, o.tx, 1, s1, w1);
    (void)w1;
    const int qx = u >= s1 ? 1 : 0;
    gen_half(G.x, o.tx, qx, s0, w0);
    int t0, h0, t1, h1;
    gen_half(G.y, o.ty, 1, t1, h1);
    (void)h1;
    const int qy = v >= t1 ? 1 : 0;
    gen_half(G.y, o.ty, qy, t0, h0);
    o.q = 2 * qy + qx;
    o.k = (v - t0) * w0 + (u - s0);
    return o;
}

// Rectangle of tiles [x0, x0 + nx) x [y0, y0 + ny).
struct GenRect {
    int32_t x0, nx, y0, ny;
};

// One phase launch.  Along each axis the tiles of index >= r are all T wide,
// so windows for halves of ceil(T/2) serve them ("narrow" blocks, blockDim
// threads each); the rows and columns of (T + 1) tiles ("wide" rectangles)
// run in the last blocks of the same launch with fewer active threads
// (n_wide, a multiple of 8 so slots stay bank-conflict free), so their larger
// windows fit the same shared memory.  One thread per (tile, lane-word group).
struct GenLaunch {
    GenRect narrow, wide[2];
    int32_t nb_narrow;  // blocks of the narrow rectangle
    int32_t n_wide;     // active threads (and slot stride) of a wide block
};

// Window slots of a thread of a narrow block.
RSOS_HD size_t gen_narrow_window_slots(const GenTiling& G)
{
    return (size_t)(((G.x.T + 1) >> 1) + 2) * (size_t)(((G.y.T + 1) >> 1) + 2);
}

// Launch plan for n threads per block and slots of wbytes bytes: the
// rectangles, the block counts, and the dynamic shared memory per block.
RSOS_HD void gen_plan_launch(const GenTiling& G, int NWP, size_t wbytes, int n, GenLaunch& P, size_t& smem,
                             long long& blocks)
{
    const int nw = (G.x.T + 1) >> 1, nh = (G.y.T + 1) >> 1;
    if (nw == G.max_w && nh == G.max_h) {
        P.narrow = GenRect{0, G.x.n, 0, G.y.n};
        P.wide[0] = P.wide[1] = GenRect{0, 0, 0, 0};
    } else {
        P.narrow = GenRect{G.x.r, G.x.n - G.x.r, G.y.r, G.y.n - G.y.r};
        P.wide[0] = GenRect{0, G.x.r, 0, G.y.n};
        P.wide[1] = GenRect{G.x.r, G.x.n - G.x.r, 0, G.y.r};
    }
    const size_t pt_narrow = gen_narrow_window_slots(G) * wbytes;
    const size_t pt_wide = (size_t)(G.max_w + 2) * (size_t)(G.max_h + 2) * wbytes;
    smem = pt_narrow * (size_t)n;
    const long long narrow_items = (long long)P.narrow.nx * P.narrow.ny * NWP;
    const long long wide_items =
        ((long long)P.wide[0].nx * P.wide[0].ny + (long long)P.wide[1].nx * P.wide[1].ny) * NWP;
    P.nb_narrow = (int32_t)((narrow_items + n - 1) / n);
    int nwide = (int)(smem / pt_wide) / 8 * 8;
    if (nwide < 8) nwide = 8;
    if (nwide > n) nwide = n;
    P.n_wide = nwide;
    if ((size_t)nwide * pt_wide > smem) smem = (size_t)nwide * pt_wide;
    blocks = P.nb_narrow + (wide_items + nwide - 1) / nwide;
}

// Tile (tx, ty), lane-word group wp and slot stride nthr of thread tid of
// block b (blockDim threads); false if the thread has no work.
RSOS_HD bool gen_item_of_thread(const GenLaunch& P, int NWP, int b, int tid, int blockDim, int& tx, int& ty, int& wp,
                                int& nthr)
{
    long long g;
    GenRect R;
    if (b < P.nb_narrow) {
        nthr = blockDim;
        g = (long long)b * nthr + tid;
        R = P.narrow;
        if (g >= (long long)R.nx * R.ny * NWP) return false;
    } else {
        nthr = P.n_wide;
        if (tid >= nthr) return false;
        g = (long long)(b - P.nb_narrow) * nthr + tid;
        R = P.wide[0];
        const long long n0 = (long long)R.nx * R.ny * NWP;
        if (g >= n0) {
            g -= n0;
            R = P.wide[1];
            if (g >= (long long)R.nx * R.ny * NWP) return false;
        }
    }
    const long long per_row = (long long)R.nx * NWP;
    const int ry = (int)(g / per_row);
    const int rem = (int)(g - (long long)ry * per_row);
    const int rx = rem / NWP;
    wp = rem - rx * NWP;
    tx = R.x0 + rx;
    ty = R.y0 + ry;
    return true;
}

}  // namespace rsos

/*
 * RSOS oracle: plain, slow CPU reference of the (2+1)-d restricted
 * solid-on-solid growth dynamics of Kelling, Odor & Gemming (arXiv:1605.02620).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link, load or call
 * this file: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg use it.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (paper section II and Eq. 6):
 *   - heights h(x,y) of an L x L periodic square lattice, flat start h = 0;
 *   - a deposition attempt at site x does h(x) -> h(x)+1 and is accepted only
 *     if afterwards |h(x) - h(n)| <= N for all four nearest neighbours n
 *     (Eq. 6).  Given the constraint already holds, this is "accept iff
 *     h(x) - h(n) < N for every neighbour n";
 *   - double tiling (DT) domain decomposition (section II): the lattice is cut
 *     into Tx x Ty tiles, each tile into 2 x 2 sub-tiles, giving four sets of
 *     sub-tiles that are updated one set after another; the tiling origin is
 *     moved randomly after every sweep; and the irregular (+1) tilings of the
 *     decomposition check (section III.C), whose tiles are T or T + 1 wide;
 *   - multisurface coding (section II): the surfaces ("lanes") of one job share
 *     the sequence of selected sites; each lane takes part in a selection only
 *     if its own random mask bit is set, so a selected site is updated in
 *     about half of the surfaces;
 *   - a true random-sequential (RS) reference dynamics: L^2 attempts at
 *     uniformly chosen sites per Monte-Carlo step;
 *   - exact sums of h and h^2 per lane, from which the squared interface width
 *     W^2 = <h^2> - <h>^2 follows (Eq. 2).
 *
 * Randomness: Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), written here from that publication.
 * The counter layout is this project's stream specification (the paper does
 * not publish one; its RNG is unnamed): key = seed, and
 *   control draw of sweep t : ctr = (0,       t, 0,      1<<30)
 *   site draws              : ctr = (tile_id, t, i>>3,   2<<30 | p<<28)
 *   mask draws              : ctr = (tile_id, t, i>>2,   3<<30 | p<<28 | w)
 *   RS site draws           : ctr = (a>>2,    s, lane,   0)
 * with t the sweep index, p the phase, i the selection index inside a
 * sub-tile activation, w = lane>>5 the 32-lane word of the lane and a the
 * attempt index inside RS step s.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Philox-4x32-10 (Salmon et al. 2011, section 4.2: the Philox S-box is a     */
/* pair of 32x32->64 multiplications whose high halves are XORed with the     */
/* other counter words and the round key; the key is advanced by a Weyl      */
/* sequence between rounds).                                                  */
/* ------------------------------------------------------------------------- */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u /* floor(2^32 * (golden ratio - 1)) */
#define ORC_PHILOX_W1 0xBB67AE85u /* floor(2^32 * (sqrt(3) - 1))      */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * x0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += ORC_PHILOX_W0;
        k1 += ORC_PHILOX_W1;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The four Philox constants (M0, M1, W0, W1), for the constant tests. */
void orc_philox_constants(uint32_t out[4])
{
    out[0] = ORC_PHILOX_M0; out[1] = ORC_PHILOX_M1;
    out[2] = ORC_PHILOX_W0; out[3] = ORC_PHILOX_W1;
}

/* n consecutive blocks: counter word 0 (carrying into word 1) runs from ctr0. */
void orc_philox_bulk(const uint32_t ctr0[4], const uint32_t key[2], uint64_t n, uint32_t* out)
{
    uint64_t base = ((uint64_t)ctr0[1] << 32) | ctr0[0];
    for (uint64_t b = 0; b < n; ++b) {
        uint64_t c01 = base + b;
        uint32_t c[4] = {(uint32_t)c01, (uint32_t)(c01 >> 32), ctr0[2], ctr0[3]};
        orc_philox4x32_10(c, key, out + 4 * b);
    }
}

/* floor(r * n / 2^32): maps a uniform 32-bit word onto [0, n). */
static uint32_t orc_mulhi32(uint32_t r, uint32_t n)
{
    return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32);
}

/* The 24 permutations of (0,1,2,3) in lexicographic order. */
static void orc_permutation(uint32_t index, int perm[4])
{
    int pool[4] = {0, 1, 2, 3};
    int n = 4;
    uint32_t fact[4] = {6, 2, 1, 1};
    for (int pos = 0; pos < 4; ++pos) {
        uint32_t pick = index / fact[pos];
        index %= fact[pos];
        perm[pos] = pool[pick];
        for (int m = (int)pick; m < n - 1; ++m) pool[m] = pool[m + 1];
        --n;
    }
}

typedef struct {
    int32_t L;           /* periodic lattice edge                              */
    int32_t N;           /* step bound of Eq. 6                                */
    int32_t Tx, Ty;      /* DT tile edges: even and dividing L (tiling 0), or  */
                         /* the base edges of a (+1) tiling (tiling 1)         */
    int32_t phase_order; /* 0: random permutation per sweep, 1: fixed 0,1,2,3  */
    int32_t tiling;      /* 0: regular Tx x Ty tiles, 1: Tx(+1) x Ty(+1) tiles  */
    uint64_t seed;       /* Philox key                                         */
} orc_params;

/* Period of the tiling pattern along an axis of edge T: T when the tiles
 * are all T wide, else the whole lattice (a (+1) tiling repeats only
 * after L sites). */
static int32_t orc_period(const orc_params* P, int32_t T)
{
    return (P->tiling == 1 && P->L % T != 0) ? P->L : T;
}

/* Control draw of sweep t: origin of the tiling, uniform over one period of
 * the pattern, and order of the four sub-tile sets (section II: the origin
 * of the decomposition moves randomly after every sweep). */
void orc_control(const orc_params* P, uint64_t t, int32_t* ox, int32_t* oy, int32_t perm[4])
{
    uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)};
    uint32_t ctr[4] = {0u, (uint32_t)t, 0u, 1u << 30};
    uint32_t r[4];
    orc_philox4x32_10(ctr, key, r);
    *ox = (int32_t)orc_mulhi32(r[0], (uint32_t)orc_period(P, P->Tx));
    *oy = (int32_t)orc_mulhi32(r[1], (uint32_t)orc_period(P, P->Ty));
    if (P->phase_order == 1) {
        for (int m = 0; m < 4; ++m) perm[m] = m;
    } else {
        orc_permutation(orc_mulhi32(r[2], 24u), perm);
    }
}

static int64_t* orc_at(int64_t* h, int32_t L, int32_t x, int32_t y)
{
    return &h[(int64_t)y * L + x];
}

/* One attempt at (x, y): Eq. 6.  Returns 1 if the deposit was accepted. */
static int orc_attempt(int64_t* h, int32_t L, int32_t N, int32_t x, int32_t y)
{
    /* periodic neighbours (0 <= x, y < L) */
    int32_t xe = x + 1 == L ? 0 : x + 1, xw = x == 0 ? L - 1 : x - 1;
    int32_t yn = y == 0 ? L - 1 : y - 1, ys = y + 1 == L ? 0 : y + 1;
    int64_t hx = *orc_at(h, L, x, y);
    int64_t nb[4] = {*orc_at(h, L, xe, y), *orc_at(h, L, xw, y),
                     *orc_at(h, L, x, yn), *orc_at(h, L, x, ys)};
    int ok = 1;
    for (int m = 0; m < 4; ++m) {
        int64_t after = hx + 1 - nb[m];
        ok &= (after <= N) & (after >= -N);
    }
    *orc_at(h, L, x, y) = hx + ok;
    return ok;
}

/* Lanes offered one selection together (lanes of one 32-lane word share
 * their mask draws; eight keep the fields a thread touches few). */
#define ORC_GROUP 8

/*
 * One activation of one sub-tile (section II): its 2a selections in order,
 * each offered to every lane of the group.  The lanes of a job share the
 * sequence of selected sites; lane j takes part in selection i only if bit
 * (j & 31) of its mask word is set (the random half mask of the multisurface
 * coding), and then makes one attempt of Eq. 6 on its own height field.
 *   x0, y0    lattice coordinates of the sub-tile's first site (taken mod L)
 *   sx, sy    extent of the sub-tile; a = sx sy
 *   fields[m] height field of lane lanes[m], m < n <= ORC_GROUP
 *   acc[m]    accepted deposits of lane m are added here
 */
static void orc_activate(const orc_params* P, int64_t* const* fields, const uint32_t* lanes, int n,
                         uint32_t tile_id, uint64_t t, int p, int32_t x0, int32_t y0, int32_t sx, int32_t sy,
                         int64_t* acc)
{
    const int32_t L = P->L;
    const uint32_t a = (uint32_t)(sx * sy);
    const uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)};
    uint32_t site_r[4], mask_r[ORC_GROUP][4];
    for (uint32_t i = 0; i < 2u * a; ++i) {
        if ((i & 7u) == 0) {
            uint32_t c[4] = {tile_id, (uint32_t)t, i >> 3, (2u << 30) | ((uint32_t)p << 28)};
            orc_philox4x32_10(c, key, site_r);
        }
        if ((i & 3u) == 0) {
            for (int m = 0; m < n; ++m) {
                if (m > 0 && (lanes[m] >> 5) == (lanes[m - 1] >> 5)) {
                    memcpy(mask_r[m], mask_r[m - 1], sizeof(mask_r[m]));  /* same word, same draw */
                    continue;
                }
                uint32_t c[4] = {tile_id, (uint32_t)t, i >> 2,
                                 (3u << 30) | ((uint32_t)p << 28) | (lanes[m] >> 5)};
                orc_philox4x32_10(c, key, mask_r[m]);
            }
        }
        uint32_t word = site_r[(i >> 1) & 3u];
        uint32_t half = (i & 1u) ? (word >> 16) : (word & 0xFFFFu);
        uint32_t k = (half * a) >> 16;
        int32_t x = (x0 + (int32_t)(k % (uint32_t)sx)) % L;
        int32_t y = (y0 + (int32_t)(k / (uint32_t)sx)) % L;
        for (int m = 0; m < n; ++m) {
            if ((mask_r[m][i & 3u] >> (lanes[m] & 31u)) & 1u) acc[m] += orc_attempt(fields[m], L, P->N, x, y);
        }
    }
}

/* The fields of lanes[g * ORC_GROUP ...] (at most ORC_GROUP of them). */
static int orc_group(int64_t* h, int64_t area, int32_t n_lanes, int32_t g, int64_t** fields)
{
    int n = n_lanes - g * ORC_GROUP;
    if (n > ORC_GROUP) n = ORC_GROUP;
    for (int m = 0; m < n; ++m) fields[m] = h + (int64_t)(g * ORC_GROUP + m) * area;
    return n;
}

/*
 * One DT sweep (sweep index t) of n_lanes height fields (section II): the
 * control draw fixes the tiling origin and the order of the four sub-tile
 * sets; then, set after set, every tile activates its sub-tile of the set.
 * The active sub-tiles of one set never touch each other's sites or halos,
 * so the method updates them concurrently: here tile rows of a set run in
 * parallel threads (each thread for one group of lanes), and the next set
 * starts when all of them are done.  accepted[m] += deposits of field m.
 */
static void orc_dt_sweep(const orc_params* P, int64_t* h, const uint32_t* lanes, int32_t n_lanes, uint64_t t,
                         int32_t n_threads, int64_t* accepted)
{
    const int32_t L = P->L, Tx = P->Tx, Ty = P->Ty;
    const int32_t sx = Tx / 2, sy = Ty / 2;
    const int32_t ntx = L / Tx, nty = L / Ty;
    const int64_t area = (int64_t)L * L;
    const int32_t groups = (n_lanes + ORC_GROUP - 1) / ORC_GROUP;
    int32_t ox, oy, perm[4];
    orc_control(P, t, &ox, &oy, perm);
    for (int p = 0; p < 4; ++p) {
        const int q = perm[p];
        const int32_t qx = q & 1, qy = q >> 1;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) num_threads(n_threads)
        for (int32_t g = 0; g < groups; ++g) {
            for (int32_t ty = 0; ty < nty; ++ty) {
                int64_t* fields[ORC_GROUP];
                int64_t acc[ORC_GROUP] = {0};
                const int n = orc_group(h, area, n_lanes, g, fields);
                for (int32_t tx = 0; tx < ntx; ++tx)
                    orc_activate(P, fields, lanes + g * ORC_GROUP, n, (uint32_t)(ty * ntx + tx), t, p,
                                 ox + tx * Tx + qx * sx, oy + ty * Ty + qy * sy, sx, sy, acc);
                for (int m = 0; m < n; ++m) {
#pragma omp atomic
                    accepted[g * ORC_GROUP + m] += acc[m];
                }
            }
        }
    }
}

/*
 * (+1) tilings (section III.C: domains of 6(+1) x 10(+1) sites).  When T does
 * not divide L, the L sites of an axis are cut into n = L div T tiles of which
 * the first r = L mod T are one site wider, so the widths add up to L (this
 * needs r <= n).  In pattern coordinates tile c starts at c T + min(c, r).
 * Every tile is halved: the first half has floor(w/2) sites, the second the
 * other w - floor(w/2), so sub-tiles of one set are always separated by a
 * half of the other set.  With T even and dividing L this is the regular
 * tiling above.
 */
typedef struct {
    int32_t T, n, r;
} orc_axis;

static orc_axis orc_axis_of(int32_t L, int32_t T)
{
    orc_axis a = {T, L / T, L % T};
    return a;
}

/* Start (pattern coordinate) and width of half `half` of tile c. */
void orc_axis_half(int32_t L, int32_t T, int32_t c, int32_t half, int32_t* start, int32_t* width)
{
    const orc_axis a = orc_axis_of(L, T);
    const int32_t X = c * a.T + (c < a.r ? c : a.r);
    const int32_t w = a.T + (c < a.r ? 1 : 0);
    const int32_t w0 = w / 2;
    *start = X + (half ? w0 : 0);
    *width = half ? w - w0 : w0;
}

/* One DT sweep of n_lanes fields on a (+1) tiling: as orc_dt_sweep, with
 * the sub-tile of tile (tx, ty) in set q spanning the halves above, a its
 * area and 2a selections per activation. */
static void orc_dt_sweep_general(const orc_params* P, int64_t* h, const uint32_t* lanes, int32_t n_lanes,
                                 uint64_t t, int32_t n_threads, int64_t* accepted)
{
    const int32_t L = P->L;
    const orc_axis ax = orc_axis_of(L, P->Tx), ay = orc_axis_of(L, P->Ty);
    const int64_t area = (int64_t)L * L;
    const int32_t groups = (n_lanes + ORC_GROUP - 1) / ORC_GROUP;
    int32_t ox, oy, perm[4];
    orc_control(P, t, &ox, &oy, perm);
    for (int p = 0; p < 4; ++p) {
        const int q = perm[p];
        const int32_t qx = q & 1, qy = q >> 1;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) num_threads(n_threads)
        for (int32_t g = 0; g < groups; ++g) {
            for (int32_t ty = 0; ty < ay.n; ++ty) {
                int64_t* fields[ORC_GROUP];
                int64_t acc[ORC_GROUP] = {0};
                const int n = orc_group(h, area, n_lanes, g, fields);
                int32_t v0, sy;
                orc_axis_half(L, P->Ty, ty, qy, &v0, &sy);
                for (int32_t tx = 0; tx < ax.n; ++tx) {
                    int32_t u0, sx;
                    orc_axis_half(L, P->Tx, tx, qx, &u0, &sx);
                    orc_activate(P, fields, lanes + g * ORC_GROUP, n, (uint32_t)(ty * ax.n + tx), t, p, ox + u0,
                                 oy + v0, sx, sy, acc);
                }
                for (int m = 0; m < n; ++m) {
#pragma omp atomic
                    accepted[g * ORC_GROUP + m] += acc[m];
                }
            }
        }
    }
}

/* One random-sequential Monte-Carlo step (L^2 attempts) of a single lane. */
static int64_t orc_rs_step_lane(const orc_params* P, int64_t* h, uint32_t lane, uint64_t s)
{
    const int32_t L = P->L;
    const uint32_t area = (uint32_t)L * (uint32_t)L;
    uint32_t key[2] = {(uint32_t)P->seed, (uint32_t)(P->seed >> 32)};
    uint32_t r[4];
    int64_t accepted = 0;
    for (uint32_t at = 0; at < area; ++at) {
        if ((at & 3u) == 0) {
            uint32_t c[4] = {at >> 2, (uint32_t)s, lane, 0u};
            orc_philox4x32_10(c, key, r);
        }
        uint32_t site = orc_mulhi32(r[at & 3u], area);
        accepted += orc_attempt(h, L, P->N, (int32_t)(site % (uint32_t)L), (int32_t)(site / (uint32_t)L));
    }
    return accepted;
}

/*
 * Advance n_lanes independent height fields by n_sweeps sweeps, starting at
 * sweep index t0.  h is [n_lanes][L][L] int64 (row-major, x fastest); lanes[m]
 * is the lane index j of field m (it selects the mask bit and mask word).
 * rs != 0 selects the random-sequential dynamics instead of DT.
 * accepted (nullable) receives the accepted deposits per field.
 * DT: the tile rows of each sub-tile set run in parallel threads (orc_dt_sweep);
 * RS: each lane is its own chain, one lane per thread.
 */
int orc_sweeps(const orc_params* P, int64_t* h, const uint32_t* lanes, int32_t n_lanes,
               uint64_t t0, uint64_t n_sweeps, int32_t rs, int32_t n_threads, int64_t* accepted)
{
    if (P->L < 1 || P->N < 1 || n_lanes < 0) return -1;
    if (P->tiling != 0 && P->tiling != 1) return -1;
    if (!rs && P->tiling == 0) {
        if (P->Tx < 2 || P->Ty < 2 || (P->Tx & 1) || (P->Ty & 1)) return -1;
        if (P->L % P->Tx || P->L % P->Ty) return -1;
    }
    if (!rs && P->tiling == 1) {
        if (P->Tx < 2 || P->Ty < 2 || P->Tx > 256 || P->Ty > 256 || P->L < P->Tx || P->L < P->Ty) return -1;
        if (P->L % P->Tx > P->L / P->Tx || P->L % P->Ty > P->L / P->Ty) return -1;
    }
    const int64_t area = (int64_t)P->L * P->L;
    if (n_threads < 1) n_threads = 1;
    int64_t* acc = (int64_t*)calloc(n_lanes > 0 ? (size_t)n_lanes : 1u, sizeof(int64_t));
    if (!acc) return -1;
    if (rs) {
        /* random-sequential steps: each lane is its own chain, one per thread */
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
        for (int32_t m = 0; m < n_lanes; ++m) {
            for (uint64_t t = t0; t < t0 + n_sweeps; ++t) acc[m] += orc_rs_step_lane(P, h + m * area, lanes[m], t);
        }
    } else {
        for (uint64_t t = t0; t < t0 + n_sweeps; ++t) {
            if (P->tiling == 1) orc_dt_sweep_general(P, h, lanes, n_lanes, t, n_threads, acc);
            else orc_dt_sweep(P, h, lanes, n_lanes, t, n_threads, acc);
        }
    }
    if (accepted) memcpy(accepted, acc, (size_t)(n_lanes > 0 ? n_lanes : 0) * sizeof(int64_t));
    free(acc);
    return 0;
}

/*
 * Exact sums of h and h^2 per field (Eq. 2 numerators), accumulated in
 * 128-bit integers.  sum_h2 is returned as (hi, lo) 64-bit halves of the
 * signed 128-bit value.
 */
void orc_sums(const int64_t* h, int32_t L, int32_t n_lanes, int64_t* sum_h,
              int64_t* sum_h2_hi, uint64_t* sum_h2_lo)
{
    const int64_t area = (int64_t)L * L;
    for (int32_t m = 0; m < n_lanes; ++m) {
        __int128 s1 = 0, s2 = 0;
        for (int64_t k = 0; k < area; ++k) {
            __int128 v = h[m * area + k];
            s1 += v;
            s2 += v * v;
        }
        sum_h[m] = (int64_t)s1;
        sum_h2_hi[m] = (int64_t)(s2 >> 64);
        sum_h2_lo[m] = (uint64_t)s2;
    }
}

/*
 * Exact power sums sum h^k, k = 1..4, per field (the raw moments behind the
 * height distribution's skewness and kurtosis, section III.C), accumulated in
 * 128-bit integers: out[8 m + 2 (k-1)] = low 64 bits, out[8 m + 2 k - 1] =
 * high 64 bits (two's complement).
 */
void orc_power_sums(const int64_t* h, int32_t L, int32_t n_lanes, int64_t* out)
{
    const int64_t area = (int64_t)L * L;
    for (int32_t m = 0; m < n_lanes; ++m) {
        __int128 s[4] = {0, 0, 0, 0};
        for (int64_t k = 0; k < area; ++k) {
            const __int128 v = h[m * area + k];
            __int128 p = v;
            for (int j = 0; j < 4; ++j) {
                s[j] += p;
                p *= v;
            }
        }
        for (int j = 0; j < 4; ++j) {
            out[8 * m + 2 * j] = (int64_t)(uint64_t)s[j];
            out[8 * m + 2 * j + 1] = (int64_t)(s[j] >> 64);
        }
    }
}

/* Largest |h(x) - h(n)| over all nearest-neighbour pairs of each field. */
void orc_max_step(const int64_t* h, int32_t L, int32_t n_lanes, int64_t* out)
{
    const int64_t area = (int64_t)L * L;
    for (int32_t m = 0; m < n_lanes; ++m) {
        const int64_t* f = h + m * area;
        int64_t best = 0;
        for (int32_t y = 0; y < L; ++y) {
            for (int32_t x = 0; x < L; ++x) {
                int64_t v = f[(int64_t)y * L + x];
                int64_t de = v - f[(int64_t)y * L + (x + 1) % L];
                int64_t ds = v - f[(int64_t)((y + 1) % L) * L + x];
                if (de < 0) de = -de;
                if (ds < 0) ds = -ds;
                if (de > best) best = de;
                if (ds > best) best = ds;
            }
        }
        out[m] = best;
    }
}

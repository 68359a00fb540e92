// Host build of the CUDA path's header-only logic (philox.cuh, rsos_logic.cuh,
// locate_origin_site) for CPU tests.  Compiled by tests/test_logic_host.py.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "philox.cuh"
#include "rsos_device.cuh"
#include "rsos_logic.cuh"
#include "rsos_geometry.h"

// One word step: residues of x and its four neighbours for 64 lanes (one
// residue per lane, values < 2^B), lane mask m; returns the accept mask and
// the new residues of x.
template <int N>
static uint64_t step_n(const int* xr, const int* er, const int* wr, const int* nr, const int* sr, uint64_t m,
                       int* xout)
{
    constexpr int B = rsos::bits_for_step(N);
    uint64_t x[B] = {}, e[B] = {}, w[B] = {}, n[B] = {}, s[B] = {};
    for (int j = 0; j < 64; ++j)
        for (int b = 0; b < B; ++b) {
            x[b] |= (uint64_t)((xr[j] >> b) & 1) << j;
            e[b] |= (uint64_t)((er[j] >> b) & 1) << j;
            w[b] |= (uint64_t)((wr[j] >> b) & 1) << j;
            n[b] |= (uint64_t)((nr[j] >> b) & 1) << j;
            s[b] |= (uint64_t)((sr[j] >> b) & 1) << j;
        }
    const uint64_t acc = rsos::accept_mask<N, B, uint64_t>(m, x, e, w, n, s);
    rsos::masked_increment<B, uint64_t>(x, acc);
    for (int j = 0; j < 64; ++j) {
        int v = 0;
        for (int b = 0; b < B; ++b) v |= (int)((x[b] >> j) & 1) << b;
        xout[j] = v;
    }
    return acc;
}

// The same step on one 128-lane word (rsos::Word128): residues of 128 lanes,
// mask in m_lo (lanes 0-63) and m_hi (64-127); acc2 receives the accept mask.
template <int N>
static void step_n128(const int* xr, const int* er, const int* wr, const int* nr, const int* sr, uint64_t m_lo,
                      uint64_t m_hi, int* xout, uint64_t* acc2)
{
    constexpr int B = rsos::bits_for_step(N);
    rsos::Word128 x[B], e[B], w[B], n[B], s[B];
    for (int b = 0; b < B; ++b) x[b] = e[b] = w[b] = n[b] = s[b] = rsos::Word128(0);
    auto set = [](rsos::Word128& v, int j, int bit) {
        if (j < 64) v.lo |= (uint64_t)bit << j;
        else v.hi |= (uint64_t)bit << (j - 64);
    };
    for (int j = 0; j < 128; ++j)
        for (int b = 0; b < B; ++b) {
            set(x[b], j, (xr[j] >> b) & 1);
            set(e[b], j, (er[j] >> b) & 1);
            set(w[b], j, (wr[j] >> b) & 1);
            set(n[b], j, (nr[j] >> b) & 1);
            set(s[b], j, (sr[j] >> b) & 1);
        }
    const rsos::Word128 acc = rsos::accept_mask<N, B, rsos::Word128>(rsos::Word128(m_lo, m_hi), x, e, w, n, s);
    rsos::masked_increment<B, rsos::Word128>(x, acc);
    for (int j = 0; j < 128; ++j) {
        int v = 0;
        for (int b = 0; b < B; ++b) v |= (int)(((j < 64 ? x[b].lo >> j : x[b].hi >> (j - 64))) & 1) << b;
        xout[j] = v;
    }
    acc2[0] = acc.lo;
    acc2[1] = acc.hi;
}

extern "C" {

void probe_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    const rsos::U4 r = rsos::philox4x32_10(rsos::U4{ctr[0], ctr[1], ctr[2], ctr[3]}, key[0], key[1]);
    out[0] = r.x; out[1] = r.y; out[2] = r.z; out[3] = r.w;
}

// n consecutive blocks from counter ctr0 (words 0-1 as one 64-bit count),
// with the round keys precomputed as the sweep kernels use them.
void probe_philox_bulk(const uint32_t* ctr0, const uint32_t* key, uint64_t n, uint32_t* out)
{
    const rsos::RoundKeys rk = rsos::philox_round_keys(key[0], key[1]);
    const uint64_t base = ((uint64_t)ctr0[1] << 32) | ctr0[0];
    for (uint64_t b = 0; b < n; ++b) {
        const uint64_t c01 = base + b;
        const rsos::U4 r = rsos::philox4x32_10(rsos::U4{(uint32_t)c01, (uint32_t)(c01 >> 32), ctr0[2], ctr0[3]}, rk);
        out[4 * b] = r.x; out[4 * b + 1] = r.y; out[4 * b + 2] = r.z; out[4 * b + 3] = r.w;
    }
}

void probe_control(uint64_t seed, uint32_t t, int T, int order, int* out6)
{
    const rsos::Control c = rsos::sweep_control((uint32_t)seed, (uint32_t)(seed >> 32), t, T, T, order);
    out6[0] = c.ox; out6[1] = c.oy;
    for (int m = 0; m < 4; ++m) out6[2 + m] = c.perm[m];
}

void probe_origin(int L, int T, int ox, int oy, int* out4)
{
    const rsos::Origin00 o = rsos::locate_origin_site(L, T, ox, oy);
    out4[0] = o.tx; out4[1] = o.ty; out4[2] = o.q; out4[3] = o.k;
}

uint64_t probe_step(int N, const int* xr, const int* er, const int* wr, const int* nr, const int* sr, uint64_t m,
                    int* xout)
{
    switch (N) {
        case 1: return step_n<1>(xr, er, wr, nr, sr, m, xout);
        case 2: return step_n<2>(xr, er, wr, nr, sr, m, xout);
        case 3: return step_n<3>(xr, er, wr, nr, sr, m, xout);
        case 4: return step_n<4>(xr, er, wr, nr, sr, m, xout);
        case 5: return step_n<5>(xr, er, wr, nr, sr, m, xout);
        case 6: return step_n<6>(xr, er, wr, nr, sr, m, xout);
        case 7: return step_n<7>(xr, er, wr, nr, sr, m, xout);
        default: return 0;
    }
}

int probe_bits(int N) { return rsos::bits_for_step(N); }

int probe_auto_tpl(int NWP, int NWT, int rows, int nT) { return rsos::auto_tiles_per_lane(NWP, NWT, rows, nT); }

void probe_step128(int N, const int* xr, const int* er, const int* wr, const int* nr, const int* sr, uint64_t m_lo,
                   uint64_t m_hi, int* xout, uint64_t* acc2)
{
    switch (N) {
        case 1: step_n128<1>(xr, er, wr, nr, sr, m_lo, m_hi, xout, acc2); break;
        case 2: step_n128<2>(xr, er, wr, nr, sr, m_lo, m_hi, xout, acc2); break;
        case 3: step_n128<3>(xr, er, wr, nr, sr, m_lo, m_hi, xout, acc2); break;
        case 4: step_n128<4>(xr, er, wr, nr, sr, m_lo, m_hi, xout, acc2); break;
        case 5: step_n128<5>(xr, er, wr, nr, sr, m_lo, m_hi, xout, acc2); break;
        case 6: step_n128<6>(xr, er, wr, nr, sr, m_lo, m_hi, xout, acc2); break;
        case 7: step_n128<7>(xr, er, wr, nr, sr, m_lo, m_hi, xout, acc2); break;
        default: break;
    }
}
}

// Scheduling rules of the persistent engine.
#include "rsos_sched.cuh"

extern "C" {

static rsos::SchedGeom make_geom(const int* g8)
{
    rsos::SchedGeom g;
    g.L = g8[0]; g.T = g8[1]; g.nT = g8[0] / g8[1]; g.K = g8[2]; g.D = g8[3]; g.phase_order = g8[4];
    g.seed_lo = (uint32_t)g8[5]; g.seed_hi = (uint32_t)g8[6];
    return g;
}

int probe_order_table(int nT, int K, int D, uint32_t* out) { return rsos::build_order_table(nT, K, D, out); }

void probe_order_entry(int nT, int K, int D, uint32_t e, int* out3)
{
    rsos::SchedGeom g{};
    g.nT = nT; g.K = K; g.D = D;
    rsos::order_entry(g, e, &out3[0], &out3[1], &out3[2]);
}

void probe_item(const int* g8, uint64_t ticket, uint32_t t0, int* out4)
{
    const rsos::Item it = rsos::item_of_ticket<0>(make_geom(g8), ticket, t0);
    out4[0] = (int)it.t; out4[1] = it.p; out4[2] = it.r; out4[3] = it.c;
}

int probe_deps(const int* g8, const int* item4, int64_t* out12)
{
    rsos::Item it;
    it.t = (uint32_t)item4[0]; it.p = item4[1]; it.r = item4[2]; it.c = item4[3];
    rsos::Dep d[4];
    const int n = rsos::item_deps<0>(make_geom(g8), it, d);
    for (int k = 0; k < n; ++k) {
        out12[3 * k] = d[k].p; out12[3 * k + 1] = d[k].r; out12[3 * k + 2] = (int64_t)d[k].target;
    }
    return n;
}
}

// Window address arithmetic of the sweep kernels (window_index) against the
// plain definition: slot (jj, ii) of the active sub-tile q of tile (tx, ty)
// holds site ((ox + tx T + qx SX + ii - 1) mod L, (oy + ty T + qy SX + jj - 1)
// mod L), whose plane-b word of lane word w is (((y T + x mod T) nT + x div T)
// B + b) NW + w.  Every combination of origin, set, tile, lane-word group,
// non-corner slot and plane is checked; returns the number of mismatches or
// out-of-range offsets and the number of checks in *n_checked.
template <int SX>
static long long window_check(int L, int NW, int B, int NWT, long long* n_checked)
{
    constexpr int T = 2 * SX;
    rsos::JobDev J{};
    J.L = L;
    J.T = T;
    J.nT = L / T;
    J.NW = NW;
    J.B = B;
    const long long total = (long long)B * L * L * NW;
    long long bad = 0, n = 0;
    for (int oy = 0; oy < T; ++oy)
        for (int ox = 0; ox < T; ++ox)
            for (int q = 0; q < 4; ++q)
                for (int ty = 0; ty < J.nT; ++ty)
                    for (int tx = 0; tx < J.nT; ++tx)
                        for (int w0 = 0; w0 + NWT <= NW; w0 += NWT) {
                            rsos::WindowIndex<SX> wi;
                            rsos::window_index<SX>(J, tx, ty, q & 1, q >> 1, ox, oy, w0, wi);
                            for (int jj = 0; jj < SX + 2; ++jj)
                                for (int ii = 0; ii < SX + 2; ++ii) {
                                    if ((jj == 0 || jj == SX + 1) && (ii == 0 || ii == SX + 1)) continue;
                                    const int x = ((ox + tx * T + (q & 1) * SX + ii - 1) % L + L) % L;
                                    const int y = ((oy + ty * T + (q >> 1) * SX + jj - 1) % L + L) % L;
                                    const long long rec = ((long long)y * T + x % T) * J.nT + x / T;
                                    for (int b = 0; b < B; ++b)
                                        for (int w = 0; w < NWT; ++w) {
                                            const long long want = (rec * B + b) * NW + w0 + w;
                                            const long long got = (long long)(wi.row[jj] + wi.col[ii]) + (long long)b * NW + w;
                                            bad += (got != want || got < 0 || got >= total) ? 1 : 0;
                                            ++n;
                                        }
                                }
                        }
    *n_checked = n;
    return bad;
}

extern "C" long long probe_window_check(int L, int T, int NW, int B, int NWT, long long* n_checked)
{
    switch (T) {
        case 2: return window_check<1>(L, NW, B, NWT, n_checked);
        case 4: return window_check<2>(L, NW, B, NWT, n_checked);
        case 8: return window_check<4>(L, NW, B, NWT, n_checked);
        case 16: return window_check<8>(L, NW, B, NWT, n_checked);
        default: return -1;
    }
}

// (+1) tilings (section III.C): geometry helpers and the window address
// arithmetic of the general phase kernel.
#include "rsos_general.cuh"

extern "C" {

void probe_gen_half(int L, int T, int c, int half, int* out2)
{
    rsos::gen_half(rsos::gen_axis(L, T), c, half, out2[0], out2[1]);
}

int probe_gen_valid(int L, int T) { return rsos::gen_axis_valid(L, T) ? 1 : 0; }

int probe_gen_period(int L, int T) { return rsos::gen_period(L, T); }

void probe_gen_locate(int L, int Tx, int Ty, int ox, int oy, int* out4)
{
    const rsos::GenOrigin o = rsos::gen_locate_origin_site(L, rsos::gen_tiling(L, Tx, Ty), ox, oy);
    out4[0] = o.tx; out4[1] = o.ty; out4[2] = o.q; out4[3] = o.k;
}

// gen_div(k, gen_inv(w)) == k / w for every w in 1..16 and k < 4096.
long long probe_gen_div_check(void)
{
    long long bad = 0;
    for (uint32_t w = 1; w <= 16; ++w)
        for (uint32_t k = 0; k < 4096; ++k) bad += rsos::gen_div(k, rsos::gen_inv(w)) != k / w;
    return bad;
}

// For every origin of one period, set q, tile and lane-word group: every
// non-corner window slot's word offset, walked as the kernel walks it
// (columns by gen_col / gen_col_next, rows by gen_row_words, plus plane b and
// word w), is in range and is the word of site ((ox + u0 + ii - 1) mod L,
// (oy + v0 + jj - 1) mod L) in the class-interleaved layout
// (((y T + x mod T) nT + x div T) B + b) NW + w with nT = ceil(L / T); the
// interior slots of the four sets cover every site exactly once; the slot
// gen_locate_origin_site names is site (0,0).  Returns the number of
// failures; *n_checked = checks made.
long long probe_gen_window_check(int L, int Tx, int Ty, int NW, int B, int NWT, long long* n_checked)
{
    const rsos::GenTiling G = rsos::gen_tiling(L, Tx, Ty);
    const int T = Tx, nT = rsos::gen_classes(L, Tx);
    const size_t rec_words = (size_t)B * NW;
    const long long total = (long long)B * L * T * nT * NW;
    const int px = rsos::gen_period(L, Tx), py = rsos::gen_period(L, Ty);
    std::vector<int> cover((size_t)L * L);
    long long bad = 0, n = 0;
    for (int oy = 0; oy < py; ++oy)
        for (int ox = 0; ox < px; ++ox) {
            std::fill(cover.begin(), cover.end(), 0);
            const rsos::GenOrigin o = rsos::gen_locate_origin_site(L, G, ox, oy);
            for (int q = 0; q < 4; ++q)
                for (int ty = 0; ty < G.y.n; ++ty)
                    for (int tx = 0; tx < G.x.n; ++tx) {
                        int u0, sw, v0, sh;
                        rsos::gen_half(G.x, tx, q & 1, u0, sw);
                        rsos::gen_half(G.y, ty, q >> 1, v0, sh);
                        rsos::GenCol col = rsos::gen_col(L, T, ox + u0 - 1);
                        for (int ii = 0; ii < sw + 2; ++ii) {
                            const size_t cw = rsos::gen_col_words(col, nT, rec_words);
                            for (int jj = 0; jj < sh + 2; ++jj) {
                                const bool edge_row = jj == 0 || jj == sh + 1, edge_col = ii == 0 || ii == sw + 1;
                                if (edge_row && edge_col) continue;
                                const int x = ((ox + u0 + ii - 1) % L + L) % L;
                                const int y = ((oy + v0 + jj - 1) % L + L) % L;
                                if (!edge_row && !edge_col) {
                                    cover[(size_t)y * L + x] += 1;
                                    const int k = (jj - 1) * sw + (ii - 1);
                                    const bool is00 = x == 0 && y == 0;
                                    const bool named = q == o.q && tx == o.tx && ty == o.ty && k == o.k;
                                    bad += is00 != named;
                                }
                                const size_t rw = rsos::gen_row_words(L, T, nT, rec_words, oy + v0 + jj - 1);
                                const long long rec = ((long long)y * T + x % T) * nT + x / T;
                                for (int w0 = 0; w0 + NWT <= NW; w0 += NWT)
                                    for (int b = 0; b < B; ++b)
                                        for (int w = 0; w < NWT; ++w) {
                                            const long long want = (rec * B + b) * NW + w0 + w;
                                            const long long got = (long long)(rw + cw) + w0 + (long long)b * NW + w;
                                            bad += (got != want || got < 0 || got >= total) ? 1 : 0;
                                            ++n;
                                        }
                            }
                            rsos::gen_col_next(col, L, T);
                        }
                    }
            for (int v : cover) bad += v != 1;
        }
    *n_checked = n;
    return bad;
}
}

extern "C" {

// Launch plan of the general phase kernel for n threads per block: every
// (tile, lane-word group) is taken by exactly one thread; every thread's
// window, for either half on both axes, lies inside the block's dynamic
// shared memory at its slot stride; slot strides are multiples of 8 (bank
// conflict free).  Returns failures; out3 = (blocks, n_wide, smem bytes).
long long probe_gen_plan_check(int L, int Tx, int Ty, int NWP, int wbytes, int n, long long* out3)
{
    const rsos::GenTiling G = rsos::gen_tiling(L, Tx, Ty);
    rsos::GenLaunch P;
    size_t smem = 0;
    long long blocks = 0;
    rsos::gen_plan_launch(G, NWP, (size_t)wbytes, n, P, smem, blocks);
    out3[0] = blocks;
    out3[1] = P.n_wide;
    out3[2] = (long long)smem;
    std::vector<int> seen((size_t)G.x.n * G.y.n * NWP);
    long long bad = 0;
    for (long long b = 0; b < blocks; ++b)
        for (int tid = 0; tid < n; ++tid) {
            int tx, ty, wp, nthr;
            if (!rsos::gen_item_of_thread(P, NWP, (int)b, tid, n, tx, ty, wp, nthr)) continue;
            if (tx < 0 || tx >= G.x.n || ty < 0 || ty >= G.y.n || wp < 0 || wp >= NWP || tid >= nthr || nthr % 8) {
                ++bad;
                continue;
            }
            seen[((size_t)ty * G.x.n + tx) * NWP + wp] += 1;
            for (int q = 0; q < 4; ++q) {
                int u0, sw, v0, sh;
                rsos::gen_half(G.x, tx, q & 1, u0, sw);
                rsos::gen_half(G.y, ty, q >> 1, v0, sh);
                const size_t last_slot = (size_t)(sw + 2) * (sh + 2) - 1;
                const size_t end = ((last_slot * nthr + tid) + 1) * (size_t)wbytes;
                bad += end > smem;
            }
        }
    for (int v : seen) bad += v != 1;
    return bad;
}
}

// Scheduling rules of the persistent engine on (+1) tilings.
#include "rsos_gen_sched.cuh"

extern "C" {

// g8: L, Tx, Ty, K, D, phase_order, seed_lo, seed_hi
static rsos::GenSchedGeom make_gen_geom(const int* g8)
{
    rsos::GenSchedGeom g;
    g.L = g8[0];
    g.y = rsos::gen_axis(g8[0], g8[2]);
    g.Px = rsos::gen_period(g8[0], g8[1]);
    g.Py = rsos::gen_period(g8[0], g8[2]);
    g.K = g8[3]; g.D = g8[4]; g.phase_order = g8[5];
    g.seed_lo = (uint32_t)g8[6]; g.seed_hi = (uint32_t)g8[7];
    return g;
}

void probe_gen_item(const int* g8, uint64_t ticket, uint32_t t0, int* out4)
{
    rsos::GenSweepCtx c;
    c.t = 0xffffffffu;
    const rsos::Item it = rsos::gen_item_of_ticket(make_gen_geom(g8), ticket, t0, &c);
    out4[0] = (int)it.t; out4[1] = it.p; out4[2] = it.r; out4[3] = it.c;
}

int probe_gen_deps(const int* g8, const int* item4, int64_t* out12)
{
    rsos::Item it;
    it.t = (uint32_t)item4[0]; it.p = item4[1]; it.r = item4[2]; it.c = item4[3];
    rsos::Dep d[4];
    const int n = rsos::gen_item_deps(make_gen_geom(g8), it, d);
    for (int k = 0; k < n; ++k) {
        out12[3 * k] = d[k].p; out12[3 * k + 1] = d[k].r; out12[3 * k + 2] = (int64_t)d[k].target;
    }
    return n;
}
}


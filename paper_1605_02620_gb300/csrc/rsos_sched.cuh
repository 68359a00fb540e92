// Work order and dependencies of the persistent dataflow engine.
//
// The double-tiling sweep (section II) is a sequence of phases; inside a
// phase all active sub-tiles are independent.  Instead of a grid-wide barrier
// after every phase, the engine splits each phase into work items
//     (t, p, r, c) = sweep t, phase p, tile row r of sweep t's tiling,
//                    chunk c of K consecutive chunks of that row,
// and lets an item start as soon as the items it conflicts with are done.  An
// item reads and writes only its sub-tiles and their one-site halos, so
//   - for p >= 1 it needs phase p-1 of rows r-1, r, r+1 of the same sweep;
//   - for p == 0 it needs phase 3 of sweep t-1 on every tile row of t-1's
//     tiling that starts less than T + 2 site rows away from its own tile row
//     (the tiling moved between the sweeps; footprints reach one site beyond
//     a tile row).
// Everything else follows transitively.  Completion is counted per (p, r):
// done[p][r] reaches (t+1)*K when every chunk of rows r in sweeps <= t is done.
//
// Tickets hand the items out in an order in which every dependency precedes
// its dependants (so the lowest unfinished ticket can always run and the
// engine cannot deadlock): sweeps in order; inside a sweep, phase p visits
// tile rows starting at s_t + p, and row j of that visit is placed at slot
// j + D*p.  The phase lag D keeps dependencies far behind the front of the
// ticket stream, so items rarely wait, while the rows touched between the
// phase-0 front and the phase-3 front (3D tile rows) stay resident in L2.
#pragma once
#include "philox.cuh"

namespace rsos {

struct SchedGeom {
    int L, T, nT;  // lattice, tile edge, tile rows
    int K;         // chunks per tile row
    int D;         // phase lag in slots
    int phase_order;
    uint32_t seed_lo, seed_hi;
};

struct Item {
    uint32_t t;
    int p, r, c;
};

struct Dep {
    int p, r;
    uint64_t target;  // done[p][r] must reach this value
};

RSOS_HD int mod_pos(int a, int n)
{
    const int m = a % n;
    return m < 0 ? m + n : m;
}

// a mod n for a in [-n, 2n): conditional adds instead of a division.
RSOS_HD int wrap1(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// Tile row where sweep t's phase 0 starts: the row holding site row 64 t
// (mod L).  Consecutive sweeps start 64 site rows apart, so a new sweep
// begins where the previous one finished its first rows long ago.
// TT > 0 is the tile edge known at compile time (g.T otherwise).
template <int TT = 0>
RSOS_HD int sweep_start_row(const SchedGeom& g, uint32_t t, int oy)
{
    const int T = TT > 0 ? TT : g.T;
    const int y = (int)((uint32_t)((uint64_t)(t % (uint32_t)g.L) * 64u % (uint32_t)g.L));
    return wrap1(y - oy, g.L) / T;
}

// Entries of one sweep's ticket order that lie in slots before s: phase p
// visits slots D p .. D p + nT - 1 with K chunks each.
RSOS_HD uint32_t entries_before_slot(const SchedGeom& g, int s)
{
    int n = 0;
    for (int p = 0; p < 4; ++p) {
        int v = s - g.D * p;
        v = v < 0 ? 0 : (v > g.nT ? g.nT : v);
        n += v;
    }
    return (uint32_t)n * (uint32_t)g.K;
}

// Slot-ordered list of (p, j, c) of one sweep: entry = p | j << 2 | c << 20.
// Host only: the reference enumeration of the order item_of_ticket computes.
// Returns the number of entries (4 * nT * K).
inline int build_order_table(int nT, int K, int D, uint32_t* out)
{
    int n = 0;
    const int slots = nT + 3 * D;
    for (int s = 0; s < slots; ++s)
        for (int p = 0; p < 4; ++p) {
            const int j = s - D * p;
            if (j < 0 || j >= nT) continue;
            for (int c = 0; c < K; ++c) out[n++] = (uint32_t)p | ((uint32_t)j << 2) | ((uint32_t)c << 20);
        }
    return n;
}

// Entry e (0 <= e < 4 nT K) of a sweep's ticket order as (p, j, c), the
// same as build_order_table's, computed without memory traffic: a binary
// search for the slot holding e, then the phase and chunk among the slot's
// entries (phases in increasing p, K chunks each).
RSOS_HD void order_entry(const SchedGeom& g, uint32_t e, int* p, int* j, int* c)
{
    const uint32_t K = (uint32_t)g.K;
    const int D = g.D, nT = g.nT;
    if (3 * D <= nT) {
        // The phase fronts enter one after another, all four run together,
        // then they leave one after another: seven segments of slots with
        // m = 1, 2, 3, 4, 3, 2, 1 phases (first phase p_lo) and m K entries each.
        // entries before segment k (in units of K): D * {0, 1, 3, 6} entering,
        // 4 nT - D * {6, 3, 1} leaving (triangular numbers)
        auto before = [&](int k) {
            return k < 4 ? (uint32_t)D * (uint32_t)(k * (k + 1) / 2)
                         : 4u * (uint32_t)nT - (uint32_t)D * (uint32_t)((7 - k) * (8 - k) / 2);
        };
        int seg = 0;
#pragma unroll
        for (int k = 1; k < 7; ++k) seg += e >= before(k) * K ? 1 : 0;
        const int m = seg < 4 ? seg + 1 : 7 - seg;
        const int p_lo = seg < 4 ? 0 : seg - 3;
        const int s0 = seg < 4 ? seg * D : nT + (seg - 4) * D;
        const uint32_t off = e - before(seg) * K;
        const uint32_t per_slot = (uint32_t)m * K;
        const uint32_t ds = off / per_slot;
        const uint32_t o = off - ds * per_slot;
        const uint32_t pi = o / K;
        *p = p_lo + (int)pi;
        *c = (int)(o - pi * K);
        *j = s0 + (int)ds - D * *p;
        return;
    }
    int lo = 0, hi = g.nT + 3 * g.D;  // entries_before_slot(lo) <= e < entries_before_slot(hi)
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (entries_before_slot(g, mid) <= e) lo = mid;
        else hi = mid;
    }
    const uint32_t o = e - entries_before_slot(g, lo);
    int p0 = 0;
    while (lo - g.D * p0 >= g.nT) ++p0;  // first phase visiting slot lo
    const uint32_t pi = o / K;
    *p = p0 + (int)pi;
    *c = (int)(o - pi * K);
    *j = lo - g.D * *p;
}

// Per-sweep quantities of the items of one sweep, computed once per sweep
// (a worker's consecutive tickets mostly share one).
struct SweepCtx {
    uint32_t t;     // sweep (0xffffffff: none yet)
    Control ctl;    // its control draw
    int start_row;  // tile row where its phase 0 starts
    int oy_prev;    // row offset of the previous sweep's tiling (t > 0)
};

template <int TT = 0>
RSOS_HD void sweep_ctx(const SchedGeom& g, uint32_t t, SweepCtx* c)
{
    const int T = TT > 0 ? TT : g.T;
    c->t = t;
    c->ctl = sweep_control(g.seed_lo, g.seed_hi, t, T, T, g.phase_order);
    c->start_row = sweep_start_row<TT>(g, t, c->ctl.oy);
    c->oy_prev = t > 0 ? sweep_control(g.seed_lo, g.seed_hi, t - 1, T, T, g.phase_order).oy : 0;
}

// Item of a ticket; tickets of one launch are 32-bit (launches are split).
// c caches the sweep's quantities and is refreshed when the sweep changes.
template <int TT = 0>
RSOS_HD Item item_of_ticket(const SchedGeom& g, uint64_t ticket, uint32_t t0, SweepCtx* c)
{
    const uint32_t per_sweep = 4u * (uint32_t)g.nT * (uint32_t)g.K;
    const uint32_t tk = (uint32_t)ticket;
    const uint32_t sw = tk / per_sweep;
    Item it;
    it.t = t0 + sw;
    if (c->t != it.t) sweep_ctx<TT>(g, it.t, c);
    int j = 0;
    order_entry(g, tk - sw * per_sweep, &it.p, &j, &it.c);
    int r = c->start_row + it.p + j;  // <= 2 nT + 1
    r = r >= g.nT ? r - g.nT : r;
    r = r >= g.nT ? r - g.nT : r;
    it.r = g.nT >= 2 ? r : 0;
    return it;
}

// Same, without a cache; returns the sweep's control draw (nullable).
template <int TT = 0>
RSOS_HD Item item_of_ticket(const SchedGeom& g, uint64_t ticket, uint32_t t0, Control* ctl_out = nullptr)
{
    SweepCtx c;
    c.t = 0xffffffffu;
    const Item it = item_of_ticket<TT>(g, ticket, t0, &c);
    if (ctl_out) *ctl_out = c.ctl;
    return it;
}

// Dependency k (0 <= k < 4) of an item, if it has one (at most four: three
// tile rows, four for T = 2 at a sweep boundary).  Each lane of a worker warp
// computes its own, in registers.  c: the item's sweep (item_of_ticket).
template <int TT = 0>
RSOS_HD bool item_dep(const SchedGeom& g, const Item& it, int k, const SweepCtx& c, Dep* out)
{
    const int T = TT > 0 ? TT : g.T;
    if (it.p > 0) {
        const uint64_t target = ((uint64_t)it.t + 1) * (uint64_t)g.K;
        if (g.nT >= 3) {
            if (k > 2) return false;
            *out = Dep{it.p - 1, wrap1(it.r + k - 1, g.nT), target};
        } else {
            if (k >= g.nT) return false;
            *out = Dep{it.p - 1, wrap1(it.r + k, g.nT), target};
        }
        return true;
    }
    if (it.t == 0 || k > 3) return false;
    // Rows r' of the previous tiling whose first site row oy_prev + r' T lies
    // in (y0 - T - 2, y0 + T + 2), y0 = first site row of this tile row: the
    // offsets y0 + dy, dy in [-(T+1), T+1], that are multiples of T from oy_prev.
    const int base = it.r * T + c.ctl.oy - c.oy_prev;  // y0 - oy_prev, in (-T, L + T)
    // smallest dy >= -(T+1) with base + dy = 0 mod T
    int dy0 = -(T + 1);
    int rem = (base + dy0) % T;
    if (rem < 0) rem += T;
    if (rem) dy0 += T - rem;
    const int dy = dy0 + k * T;
    if (dy > T + 1) return false;
    // (base + dy) / T is in [-2, nT + 2): exact division, wrapped by additions
    auto row_of = [&](int d) {
        int r = (base + d) / T;
        r = r < 0 ? r + g.nT : r;
        r = r >= g.nT ? r - g.nT : r;
        r = r < 0 ? r + g.nT : r;
        return r >= g.nT ? r - g.nT : r;
    };
    const int r = row_of(dy);
    for (int k2 = 0; k2 < k; ++k2)  // rows already covered by an earlier dependency
        if (row_of(dy0 + k2 * T) == r) return false;
    *out = Dep{3, r, (uint64_t)it.t * (uint64_t)g.K};
    return true;
}

// Same, computing the sweep's quantities itself (host tests).
template <int TT = 0>
RSOS_HD bool item_dep(const SchedGeom& g, const Item& it, int k, Dep* out)
{
    SweepCtx c;
    sweep_ctx<TT>(g, it.t, &c);
    return item_dep<TT>(g, it, k, c, out);
}

// All dependencies of an item, packed (host tests).
template <int TT = 0>
RSOS_HD int item_deps(const SchedGeom& g, const Item& it, Dep* out)
{
    int n = 0;
    for (int k = 0; k < 4; ++k) {
        Dep d;
        if (item_dep<TT>(g, it, k, &d)) out[n++] = d;
    }
    return n;
}

}  // namespace rsos

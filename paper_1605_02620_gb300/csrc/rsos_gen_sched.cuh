// Work order and dependencies of the persistent engine on the (+1) tilings
// of the decomposition check (section III.C).
//
// Items (t, p, r, c), tickets and phase fronts are those of rsos_sched.cuh,
// with r a tile row of sweep t's tiling: ny rows along y, T or T + 1 sites
// high, and K chunks of the nx tiles of a row.  Phases p >= 1 depend, as
// there, on phase p - 1 of rows r - 1, r, r + 1 of the same sweep: a
// sub-tile and its one-site halo lie in its own tile row and the rows next
// to it.  What changes is phase 0: the origin of the tiling moves anywhere
// in the period of the pattern between sweeps (the whole lattice when T
// does not divide L), so phase 0 of row r depends on phase 3 of sweep t - 1
// on every row of the previous tiling that meets tile row r grown by one
// halo site above and below: at most four rows (T = 2: a window of five
// sites over rows at least two high), three for T >= 3.
#pragma once
#include "philox.cuh"
#include "rsos_general.cuh"
#include "rsos_sched.cuh"

namespace rsos {

struct GenSchedGeom {
    int L;
    GenAxis y;   // the tile rows: n rows, the first r of them T + 1 high
    int Px, Py;  // periods of the origin draw along x and y
    int K, D, phase_order;
    uint32_t seed_lo, seed_hi;
};

// The ticket order's geometry: order_entry depends only on the number of
// rows, the chunks per row and the phase lag.
RSOS_HD SchedGeom gen_order_geom(const GenSchedGeom& g)
{
    SchedGeom s{};
    s.L = g.L;
    s.T = g.y.T;
    s.nT = g.y.n;
    s.K = g.K;
    s.D = g.D;
    s.phase_order = g.phase_order;
    s.seed_lo = g.seed_lo;
    s.seed_hi = g.seed_hi;
    return s;
}

// First pattern row of tile row r and its height.
RSOS_HD void gen_row_span(const GenAxis& a, int r, int& start, int& height)
{
    start = r * a.T + (r < a.r ? r : a.r);
    height = a.T + (r < a.r ? 1 : 0);
}

// Per-sweep quantities, refreshed when a worker's sweep changes.
struct GenSweepCtx {
    uint32_t t;     // sweep (0xffffffff: none yet)
    Control ctl;    // its control draw (origin over one period, phase order)
    int start_row;  // tile row where its phase 0 starts
    int oy_prev;    // row offset of the previous sweep's tiling (t > 0)
};

RSOS_HD void gen_sweep_ctx(const GenSchedGeom& g, uint32_t t, GenSweepCtx* c)
{
    c->t = t;
    c->ctl = sweep_control(g.seed_lo, g.seed_hi, t, g.Px, g.Py, g.phase_order);
    // the tile row holding site row 64 t (mod L), as the regular engine does
    const int y = (int)((uint32_t)((uint64_t)(t % (uint32_t)g.L) * 64u % (uint32_t)g.L));
    c->start_row = gen_tile_of(g.y, gen_wrap(y - c->ctl.oy, g.L));
    c->oy_prev = t > 0 ? sweep_control(g.seed_lo, g.seed_hi, t - 1, g.Px, g.Py, g.phase_order).oy : 0;
}

// Item of a ticket (tickets of one launch are 32-bit); c caches the sweep.
RSOS_HD Item gen_item_of_ticket(const GenSchedGeom& g, uint64_t ticket, uint32_t t0, GenSweepCtx* c)
{
    const int ny = g.y.n;
    const uint32_t per_sweep = 4u * (uint32_t)ny * (uint32_t)g.K;
    const uint32_t tk = (uint32_t)ticket;
    const uint32_t sw = tk / per_sweep;
    Item it;
    it.t = t0 + sw;
    if (c->t != it.t) gen_sweep_ctx(g, it.t, c);
    int j = 0;
    order_entry(gen_order_geom(g), tk - sw * per_sweep, &it.p, &j, &it.c);
    int r = c->start_row + it.p + j;  // <= 2 ny + 1
    r = r >= ny ? r - ny : r;
    r = r >= ny ? r - ny : r;
    it.r = ny >= 2 ? r : 0;
    return it;
}

// Dependency k (0 <= k < 4) of an item, if it has one.  c: the item's sweep.
RSOS_HD bool gen_item_dep(const GenSchedGeom& g, const Item& it, int k, const GenSweepCtx& c, Dep* out)
{
    const int ny = g.y.n;
    if (it.p > 0) {
        const uint64_t target = ((uint64_t)it.t + 1) * (uint64_t)g.K;
        if (ny >= 3) {
            if (k > 2) return false;
            *out = Dep{it.p - 1, wrap1(it.r + k - 1, ny), target};
        } else {
            if (k >= ny) return false;
            *out = Dep{it.p - 1, wrap1(it.r + k, ny), target};
        }
        return true;
    }
    if (it.t == 0 || k > 3) return false;
    // Site rows of tile row r with one halo row on each side, as pattern
    // rows of the previous tiling: [a, a + h + 1] with a in [0, L).
    int start, h;
    gen_row_span(g.y, it.r, start, h);
    const int a = gen_wrap(gen_wrap(start - 1 + c.ctl.oy, g.L) - c.oy_prev, g.L);
    const int first = gen_tile_of(g.y, a);
    int s0, h0;
    gen_row_span(g.y, first, s0, h0);
    // row first + k of the previous tiling starts at s0 plus the heights of
    // the rows before it (past the wrap at L the pattern repeats)
    int s = s0;
    for (int m = 0; m < k; ++m) {
        int sm, hm;
        gen_row_span(g.y, (first + m) % ny, sm, hm);
        s += hm;
    }
    if (k > 0 && s > a + h + 1) return false;  // beyond the window
    if (k >= ny) return false;                 // every row already listed
    *out = Dep{3, (first + k) % ny, (uint64_t)it.t * (uint64_t)g.K};
    return true;
}

// All dependencies of an item, computing the sweep's quantities itself (host tests).
RSOS_HD int gen_item_deps(const GenSchedGeom& g, const Item& it, Dep* out)
{
    GenSweepCtx c;
    gen_sweep_ctx(g, it.t, &c);
    int n = 0;
    for (int k = 0; k < 4; ++k) {
        Dep d;
        if (gen_item_dep(g, it, k, c, &d)) out[n++] = d;
    }
    return n;
}

}  // namespace rsos

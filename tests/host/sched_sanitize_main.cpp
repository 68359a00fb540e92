// Test driver: the persistent engine's host-compiled scheduling arithmetic
// (ticket -> item, dependencies, per-sweep context) over many geometries,
// built with the host address and undefined-behaviour sanitizers.
#include <cstdio>
#include <vector>

#include "rsos_sched.cuh"

int main()
{
    unsigned long long check = 0;
    const int geoms[][4] = {{32, 8, 2, 2}, {64, 8, 4, 7}, {16, 2, 8, 3}, {4096, 8, 8, 170}, {256, 4, 2, 40}, {8, 8, 1, 2}};
    for (const auto& gm : geoms) {
        rsos::SchedGeom g{};
        g.L = gm[0];
        g.T = gm[1];
        g.nT = gm[0] / gm[1];
        g.K = gm[2];
        g.D = gm[3];
        g.phase_order = 0;
        g.seed_lo = 77;
        g.seed_hi = 3;
        std::vector<uint32_t> table((size_t)4 * g.nT * g.K);
        if (rsos::build_order_table(g.nT, g.K, g.D, table.data()) != (int)table.size()) return 1;
        rsos::SweepCtx c;
        c.t = 0xffffffffu;
        const uint64_t n = 3 * table.size();
        for (uint64_t tk = 0; tk < n; tk += 1 + tk / 1000) {
            const rsos::Item it = rsos::item_of_ticket<0>(g, tk, 5u, &c);
            for (int k = 0; k < 4; ++k) {
                rsos::Dep d;
                if (rsos::item_dep<0>(g, it, k, c, &d)) {
                    if (d.r < 0 || d.r >= g.nT || d.p < 0 || d.p > 3) return 2;
                    check = check * 131u + (unsigned long long)d.r + d.target;
                }
            }
            check = check * 31u + (unsigned long long)it.r + (unsigned long long)it.c * 7u + (unsigned long long)it.p;
        }
    }
    std::printf("%llu\n", check);
    return 0;
}

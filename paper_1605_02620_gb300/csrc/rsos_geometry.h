// Automatic work-item size of the persistent engine (execution geometry
// only: results are bit-identical for every choice).  Plain host/device
// arithmetic, shared by the library and its CPU tests.
#pragma once
#include "rsos_common.cuh"

namespace rsos {

// Work items of one phase of one sweep (tile rows x chunks per row) that
// keep the persistent engine's workers (152 SMs x 12 warps = 1824 on GB300)
// busy between the phase fronts: twice the workers.
constexpr long long kMinItemsPerPhase = 2 * 152 * 12;

// Tiles per lane of a job without an explicit choice:
// * several lane-word groups per tile (NWP > 1): 2 per group, at most 8;
// * one word group per lane: the largest power of two from 2 up that leaves
//   at least kMinItemsPerPhase items per phase (rows tile rows, nT tiles per
//   row, 32 lanes per item), at most 16 for 32-bit words (NWT = 1) and 4 for
//   wider ones.  A larger item spreads its fixed costs (ticket, dependency
//   waits, completion) over more tiles, as long as enough items remain to
//   keep every worker busy.  Measured on GB300, us per sweep: L = 4096: 2 per
//   lane (4096 items per phase) fastest for 32- and 64-bit words, 4 (2048
//   items) 4-8% slower; L = 8192, 32 surfaces: 2 / 4 / 8 per lane 410 / 381 /
//   368 (8: 4096 items); 64 surfaces: 2 / 4 per lane 589 / 563; L = 32768,
//   32 surfaces, N = 1: 2 / 8 / 16 per lane 6537 / 5806 / 5680, N = 4:
//   9067 / 8477 / 8385; (+1) tilings, L = 9605, 6(+1) x 10(+1), 64
//   surfaces: 1 / 2 / 4 / 8 per lane 1489 / 1374 / 1324 / 1327 (4: 12480
//   items).
RSOS_HD int auto_tiles_per_lane(int NWP, int NWT, int rows, int nT)
{
    if (NWP > 1) return NWP <= 4 ? 2 * NWP : 8;
    int tpl = 2;
    const int cap = NWT == 1 ? 16 : 4;
    while (tpl < cap) {
        const long long item = 32LL * 2 * tpl;  // tiles of an item at twice the tiles per lane
        const long long k = (nT + item - 1) / item;
        if ((long long)rows * k < kMinItemsPerPhase) break;
        tpl *= 2;
    }
    return tpl;
}

}  // namespace rsos

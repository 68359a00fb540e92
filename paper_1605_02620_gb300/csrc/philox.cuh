// Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two
// 32x32->64 multiplications whose high halves are mixed into the other
// counter words with the round key; the key advances by a Weyl sequence.
//
// The RSOS method (section II) only needs "random" site selections, half
// masks and tiling origins; this stateless generator replaces the per-thread
// RNG states the paper mentions, so any item of work can be recomputed from
// (seed, sweep, phase, tile, selection, lane word) alone.
#pragma once
#include "rsos_common.cuh"

namespace rsos {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;  // golden-ratio Weyl increment
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;  // sqrt(3)-1 Weyl increment

// One 32x32->64 multiply gives both halves.
RSOS_HD void mul_hi_lo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo)
{
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    lo = (uint32_t)p;
    hi = (uint32_t)(p >> 32);
}

RSOS_HD U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mul_hi_lo(kPhiloxM0, c.x, hi0, lo0);
        mul_hi_lo(kPhiloxM1, c.z, hi1, lo1);
        const U4 n = {hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        c = n;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return c;
}

// Round keys of one Philox key: k[2r], k[2r+1] are the key words used in
// round r.  Precomputed once per job so a block evaluates the generator with
// the keys as uniform kernel-parameter operands.
struct RoundKeys {
    uint32_t k[20];
};

RSOS_HD RoundKeys philox_round_keys(uint32_t k0, uint32_t k1)
{
    RoundKeys rk;
    for (int r = 0; r < 10; ++r) {
        rk.k[2 * r] = k0;
        rk.k[2 * r + 1] = k1;
        k0 += kPhiloxW0;
        k1 += kPhiloxW1;
    }
    return rk;
}

RSOS_HD U4 philox4x32_10(U4 c, const RoundKeys& rk)
{
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mul_hi_lo(kPhiloxM0, c.x, hi0, lo0);
        mul_hi_lo(kPhiloxM1, c.z, hi1, lo1);
        const U4 n = {hi1 ^ c.y ^ rk.k[2 * r], lo1, hi0 ^ c.w ^ rk.k[2 * r + 1], lo0};
        c = n;
    }
    return c;
}

// floor(r * n / 2^32)
RSOS_HD uint32_t scale32(uint32_t r, uint32_t n)
{
    return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32);
}

// Per-sweep control draw: tiling origin (ox, oy) in [0,Tx) x [0,Ty) and the
// order in which the four sub-tile sets are visited (section II: the origin of
// the decomposition moves randomly after every sweep).
struct Control {
    int ox, oy;
    int perm[4];
};

RSOS_HD Control sweep_control(uint32_t seed_lo, uint32_t seed_hi, uint32_t t, int Tx, int Ty,
                              int phase_order)
{
    const U4 r = philox4x32_10(U4{0u, t, 0u, kDomControl}, seed_lo, seed_hi);
    Control c;
    c.ox = (int)scale32(r.x, (uint32_t)Tx);
    c.oy = (int)scale32(r.y, (uint32_t)Ty);
    if (phase_order == 1) {
        for (int m = 0; m < 4; ++m) c.perm[m] = m;
        return c;
    }
    // Lexicographic rank -> permutation (factorial number system).
    uint32_t rank = scale32(r.z, 24u);
    int avail = 0xF;  // bit set of unused sub-tile sets
    const uint32_t radix[4] = {6u, 2u, 1u, 1u};
    for (int m = 0; m < 4; ++m) {
        uint32_t pick = rank / radix[m];
        rank -= pick * radix[m];
        int v = 0;
        for (;; ++v) {
            if (avail & (1 << v)) {
                if (pick == 0) break;
                --pick;
            }
        }
        c.perm[m] = v;
        avail &= ~(1 << v);
    }
    return c;
}

}  // namespace rsos

// Shared definitions of the CUDA path (device and host code of librsos).
#pragma once
#include <stddef.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define RSOS_HD __host__ __device__ __forceinline__
#else
#define RSOS_HD inline
#endif

namespace rsos {

struct U4 {
    uint32_t x, y, z, w;
};

// Stream domains (top two bits of counter word 3).
constexpr uint32_t kDomControl = 1u << 30;
constexpr uint32_t kDomSite = 2u << 30;
constexpr uint32_t kDomMask = 3u << 30;

// Bits per site and surface needed to code every neighbour difference in
// [-N, N] losslessly as h mod 2^B: 2^B >= 2N + 1.
RSOS_HD constexpr int bits_for_step(int N) { return N <= 1 ? 2 : (N <= 3 ? 3 : 4); }

// A 128-lane storage word: four consecutive 32-lane words of one bit plane,
// lanes 0-63 in lo and 64-127 in hi (the little-endian order of the words in
// memory).  It carries the lane-wise operators the bit-sliced word logic
// uses, so that logic runs unchanged on 128 lanes.  Word128(0) is all zero.
struct alignas(16) Word128 {
    unsigned long long lo, hi;
    Word128() = default;
    RSOS_HD constexpr explicit Word128(int v) : lo((unsigned long long)(unsigned)v), hi(0ull) {}
    RSOS_HD constexpr Word128(unsigned long long l, unsigned long long h) : lo(l), hi(h) {}
};

RSOS_HD Word128 operator~(const Word128& a) { return Word128(~a.lo, ~a.hi); }
RSOS_HD Word128 operator&(const Word128& a, const Word128& b) { return Word128(a.lo & b.lo, a.hi & b.hi); }
RSOS_HD Word128 operator|(const Word128& a, const Word128& b) { return Word128(a.lo | b.lo, a.hi | b.hi); }
RSOS_HD Word128 operator^(const Word128& a, const Word128& b) { return Word128(a.lo ^ b.lo, a.hi ^ b.hi); }
RSOS_HD Word128& operator&=(Word128& a, const Word128& b) { return a = a & b; }
RSOS_HD Word128& operator|=(Word128& a, const Word128& b) { return a = a | b; }
RSOS_HD Word128& operator^=(Word128& a, const Word128& b) { return a = a ^ b; }

}  // namespace rsos

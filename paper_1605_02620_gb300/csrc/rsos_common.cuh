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

}  // namespace rsos

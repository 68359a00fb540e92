// Bit-sliced word logic of the RSOS update (Eq. 6) on multisurface-coded
// sites (section II).
//
// A site of a multisurface word W (32 or 64 lanes) holds h mod 2^B of every
// lane in B bit planes x[0..B-1] (bit j of plane b = bit b of lane j's
// residue).  Because |h(x) - h(n)| <= N and 2^B >= 2N + 1, the residues code
// every neighbour difference losslessly.  A deposit at x is rejected exactly
// when some neighbour n has h(n) = h(x) - N, i.e. when the residues satisfy
// n == x - N (mod 2^B); it is then applied as a masked ripple increment.
#pragma once
#include "rsos_common.cuh"

namespace rsos {

// y = x - C (mod 2^B), plane-wise ripple subtraction of a constant.
template <int B, int C, typename W>
RSOS_HD void sub_const(const W (&x)[B], W (&y)[B])
{
    W borrow = W(0);
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int b = 0; b < B; ++b) {
        if ((C >> b) & 1) {
            y[b] = ~(x[b] ^ borrow);
            borrow = ~x[b] | borrow;
        } else {
            y[b] = x[b] ^ borrow;
            borrow = ~x[b] & borrow;
        }
    }
}

// Lanes where the residues of n and y differ.
template <int B, typename W>
RSOS_HD W differs(const W (&n)[B], const W (&y)[B])
{
    W d = n[0] ^ y[0];
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int b = 1; b < B; ++b) d |= n[b] ^ y[b];
    return d;
}

// Lanes of `mask` whose deposit at x is allowed by Eq. 6 given the four
// neighbours e, w, n, s.
template <int N, int B, typename W>
RSOS_HD W accept_mask(W mask, const W (&x)[B], const W (&e)[B], const W (&w)[B], const W (&n)[B],
                      const W (&s)[B])
{
    W y[B];
    sub_const<B, N>(x, y);
    return mask & differs<B>(e, y) & differs<B>(w, y) & differs<B>(n, y) & differs<B>(s, y);
}

// x += acc (mod 2^B) lane-wise.
template <int B, typename W>
RSOS_HD void masked_increment(W (&x)[B], W acc)
{
    W carry = acc;
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int b = 0; b < B; ++b) {
        const W nb = x[b] ^ carry;
        carry = x[b] & carry;
        x[b] = nb;
    }
}

}  // namespace rsos

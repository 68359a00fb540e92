"""Pins for the oracle's Philox-4x32-10 (Salmon et al., SC'11).

The generator's authors publish known-answer vectors with their reference
implementation (tests/golden/philox4x32_10_kat.txt); they fix the
multipliers, the Weyl constants, the round count and the order of the four
output words.  The Weyl constants also have closed forms in that publication
(golden ratio and sqrt(3)), and the output must look like independent fair
bits.  The GPU suite additionally compares the oracle with cuRAND's device
Philox.
"""
import math
import os

import numpy as np

import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")


def read_kat(path=GOLDEN):
    """(counter[4], key[2], expected[4]) per line of the known-answer file."""
    out = []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            words = [int(w, 16) for w in line]
            assert len(words) == 10, line
            out.append((words[0:4], words[4:6], words[6:10]))
    return out


def pi_words(n):
    """First n 32-bit words of the fractional part of pi, from Machin's
    formula pi = 16 atan(1/5) - 4 atan(1/239) in fixed-point integers."""
    bits = 32 * n + 64  # guard bits
    one = 1 << bits

    def atan_inv(x):
        total, term, k, x2 = 0, one // x, 1, x * x
        while term:
            total += term // k if (k // 2) % 2 == 0 else -(term // k)
            term //= x2
            k += 2
        return total

    pi = 16 * atan_inv(5) - 4 * atan_inv(239)
    frac = (pi - 3 * one) >> 64
    return [(frac >> (32 * (n - 1 - i))) & 0xFFFFFFFF for i in range(n)]


def test_published_known_answer_vectors():
    kat = read_kat()
    assert len(kat) == 3
    for ctr, key, expected in kat:
        got = [int(v) for v in O.philox4x32_10(ctr, key)]
        assert got == expected, ([hex(v) for v in got], [hex(v) for v in expected])


def test_third_vector_inputs_are_the_digits_of_pi():
    ctr, key, _ = read_kat()[2]
    assert ctr + key == pi_words(6)


def test_weyl_constants_closed_form():
    m0, m1, w0, w1 = O.philox_constants()
    # floor(2^32 * (phi - 1)) with phi - 1 = (sqrt(5) - 1) / 2
    s5 = math.isqrt(5 << 64)
    assert w0 == (s5 - (1 << 32)) // 2
    # floor(2^32 * (sqrt(3) - 1))
    assert w1 == math.isqrt(3 << 64) - (1 << 32)
    # the multipliers are odd (invertible mod 2^32), as the construction needs
    assert m0 & 1 and m1 & 1


def test_rounds_are_bijective_on_counter():
    # distinct counters under one key give distinct blocks (Philox is a keyed
    # bijection); a dropped or duplicated counter word would collide here.
    out = O.philox_bulk([0, 0, 7, 9], [123, 456], 1 << 16)
    as_bytes = out.view(np.uint8).reshape(len(out), 16)
    assert len({bytes(r) for r in as_bytes}) == len(out)
    assert np.array_equal(O.philox4x32_10([0, 0, 7, 9], [123, 456]), out[0])
    # changing counter words 2 and 3 or either key word changes every block
    for c2, c3, k0, k1 in [(8, 9, 123, 456), (7, 10, 123, 456), (7, 9, 124, 456), (7, 9, 123, 457)]:
        alt = O.philox_bulk([0, 0, c2, c3], [k0, k1], 256)
        assert not np.any(np.all(alt == out[:256], axis=1))


def test_bit_frequencies():
    out = O.philox_bulk([0, 0, 0, 0], [0xDEADBEEF, 0x12345678], 1 << 16).ravel()
    bits = ((out[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.float64)
    n = len(out)
    freq = bits.mean(axis=0)
    sigma = 0.5 / math.sqrt(n)
    assert np.all(np.abs(freq - 0.5) < 5 * sigma), freq
    # byte histogram chi-square, 255 degrees of freedom
    hist = np.bincount(out.view(np.uint8), minlength=256).astype(np.float64)
    exp = hist.sum() / 256
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert 150 < chi2 < 380, chi2
    # lag-1 correlation of consecutive words, as uniforms
    u = out.astype(np.float64) / 2 ** 32
    c = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(c) < 5 / math.sqrt(n), c


def test_avalanche():
    rng = np.random.Generator(np.random.PCG64(1))
    flips = []
    for _ in range(200):
        ctr = rng.integers(0, 2 ** 32, size=4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
        base = O.philox4x32_10(ctr, key)
        bit = int(rng.integers(0, 128))
        c2 = ctr.copy()
        c2[bit // 32] ^= np.uint32(1 << (bit % 32))
        alt = O.philox4x32_10(c2, key)
        flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, alt)))
    assert 60 < np.mean(flips) < 68

"""Pins for the oracle's Philox-4x32-10 (Salmon et al., SC'11).

The Weyl constants have closed forms in that publication (golden ratio and
sqrt(3)); the generator's output must look like independent fair bits.  The
GPU suite additionally compares the oracle with cuRAND's device Philox.
"""
import math

import numpy as np

import oracle as O


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

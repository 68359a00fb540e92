"""CPU checks of the CUDA path's header-only logic, compiled for the host.

* the bit-sliced accept test and masked increment equal Eq. 6 applied lane by
  lane, exhaustively over every legal neighbourhood for N = 1..7;
* the device Philox and per-sweep control draw agree with the oracle's
  independent implementation (the two share no code);
* the location of site (0,0) in a shifted tiling.
"""
import ctypes
import itertools
import os
import subprocess

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1605_02620_gb300", "csrc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("probe") / "logic_probe.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", CSRC,
                           os.path.join(HERE, "host", "logic_probe.cpp"), "-o", out])
    lib = ctypes.CDLL(out)
    ip = ctypes.POINTER(ctypes.c_int)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.probe_philox.argtypes = [u32p, u32p, u32p]
    lib.probe_control.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ip]
    lib.probe_origin.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip]
    lib.probe_step.argtypes = [ctypes.c_int, ip, ip, ip, ip, ip, ctypes.c_uint64, ip]
    lib.probe_step.restype = ctypes.c_uint64
    lib.probe_bits.restype = ctypes.c_int
    return lib


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


@pytest.mark.parametrize("N", range(1, 8))
def test_word_logic_exhaustive(probe, N):
    B = probe.probe_bits(N)
    assert 2 ** B >= 2 * N + 1 and 2 ** (B - 1) < 2 * N + 1
    M = 2 ** B
    rng = np.random.Generator(np.random.PCG64(N))
    # every (h_x mod 2^B, d_E, d_W, d_N, d_S) with d in [-N, N]
    cases = np.array([(hx,) + d for hx in range(M)
                      for d in itertools.product(range(-N, N + 1), repeat=4)], dtype=np.int64)
    pad = (-len(cases)) % 64
    cases = np.concatenate([cases, cases[:pad]])
    for chunk in cases.reshape(-1, 64, 5):
        hx = chunk[:, 0]
        nb = [(hx + chunk[:, 1 + k]) % M for k in range(4)]
        for m in (0xFFFFFFFFFFFFFFFF, int(rng.integers(0, 2 ** 63)) * 2 + 1):
            xin = np.ascontiguousarray(hx, dtype=np.int32)
            args = [np.ascontiguousarray(v, dtype=np.int32) for v in nb]
            xout = np.zeros(64, dtype=np.int32)
            acc = probe.probe_step(N, _ip(xin), *[_ip(a) for a in args], m, _ip(xout))
            for j in range(64):
                # Eq. 6: after the deposit every |h(x)+1 - h(n)| <= N
                ok = all(abs(1 - chunk[j, 1 + k]) <= N for k in range(4))
                want = bool((m >> j) & 1) and ok
                assert bool((acc >> j) & 1) == want
                assert xout[j] == ((hx[j] + 1) % M if want else hx[j])


@pytest.mark.parametrize("N", range(1, 8))
def test_word_logic_exhaustive_128_lanes(probe, N):
    """The same cases on one 128-lane word (the lane-wise operators of
    Word128, used by words_per_thread = 4): every lane, in both halves,
    follows Eq. 6 and the masked increment."""
    ip = ctypes.POINTER(ctypes.c_int)
    probe.probe_step128.argtypes = [ctypes.c_int, ip, ip, ip, ip, ip, ctypes.c_uint64, ctypes.c_uint64, ip,
                                    ctypes.POINTER(ctypes.c_uint64)]
    probe.probe_step128.restype = None
    B = probe.probe_bits(N)
    M = 2 ** B
    rng = np.random.Generator(np.random.PCG64(100 + N))
    cases = np.array([(hx,) + d for hx in range(M)
                      for d in itertools.product(range(-N, N + 1), repeat=4)], dtype=np.int64)
    cases = np.concatenate([cases, cases[:(-len(cases)) % 128]])
    lanes = range(128)
    for chunk in cases.reshape(-1, 128, 5):
        hx = chunk[:, 0]
        nb = [np.ascontiguousarray((hx + chunk[:, 1 + k]) % M, dtype=np.int32) for k in range(4)]
        ok = np.all(np.abs(1 - chunk[:, 1:]) <= N, axis=1)
        for m_lo, m_hi in ((2 ** 64 - 1, 2 ** 64 - 1),
                           (int(rng.integers(0, 2 ** 63)) * 2 + 1, int(rng.integers(0, 2 ** 63)))):
            xin = np.ascontiguousarray(hx, dtype=np.int32)
            xout = np.zeros(128, dtype=np.int32)
            acc = np.zeros(2, dtype=np.uint64)
            probe.probe_step128(N, _ip(xin), *[_ip(a) for a in nb], m_lo, m_hi, _ip(xout),
                                acc.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
            mask = np.array([(m_lo >> j) & 1 if j < 64 else (m_hi >> (j - 64)) & 1 for j in lanes], dtype=bool)
            want = mask & ok
            got = np.array([(int(acc[0]) >> j) & 1 if j < 64 else (int(acc[1]) >> (j - 64)) & 1 for j in lanes],
                           dtype=bool)
            assert np.array_equal(got, want)
            assert np.array_equal(xout, np.where(want, (hx + 1) % M, hx))

def test_device_philox_matches_oracle(probe):
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(2000):
        ctr = rng.integers(0, 2 ** 32, size=4, dtype=np.uint64).astype(np.uint32)
        key = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
        out = np.zeros(4, dtype=np.uint32)
        u32 = ctypes.POINTER(ctypes.c_uint32)
        probe.probe_philox(ctr.ctypes.data_as(u32), key.ctypes.data_as(u32), out.ctypes.data_as(u32))
        assert np.array_equal(out, O.philox4x32_10(ctr, key))


def test_device_philox_matches_oracle_on_a_million_blocks(probe):
    """The device Philox (round keys precomputed, as the kernels use it) and
    the oracle's independent one agree on 10^6 blocks: 1000 random keys x
    1000 consecutive counters from random starts (including carries into the
    high counter word)."""
    u32 = ctypes.POINTER(ctypes.c_uint32)
    probe.probe_philox_bulk.argtypes = [u32, u32, ctypes.c_uint64, u32]
    rng = np.random.Generator(np.random.PCG64(6))
    for k in range(1000):
        key = rng.integers(0, 2 ** 32, size=2, dtype=np.uint64).astype(np.uint32)
        ctr = rng.integers(0, 2 ** 32, size=4, dtype=np.uint64).astype(np.uint32)
        if k % 10 == 0:
            ctr[0] = 2 ** 32 - 300  # the 64-bit count carries into word 1
        got = np.zeros((1000, 4), dtype=np.uint32)
        probe.probe_philox_bulk(ctr.ctypes.data_as(u32), key.ctypes.data_as(u32), 1000, got.ctypes.data_as(u32))
        assert np.array_equal(got, O.philox_bulk(ctr, key, 1000)), k


@pytest.mark.parametrize("T,order", [(8, 0), (2, 0), (16, 1), (4, 0)])
def test_device_control_matches_oracle(probe, T, order):
    seed = 0xABCDEF0123456789
    p = O.Params(L=64, N=1, Tx=T, Ty=T, phase_order=order, seed=seed)
    out = np.zeros(6, dtype=np.int32)
    for t in range(0, 5000, 7):
        probe.probe_control(seed, t, T, order, _ip(out))
        ox, oy, perm = O.control(p, t)
        assert (out[0], out[1], tuple(out[2:])) == (ox, oy, perm)


def test_origin_site_location(probe):
    out = np.zeros(4, dtype=np.int32)
    for L, T in [(64, 8), (16, 4), (2, 2), (48, 16)]:
        S = T // 2
        for ox in range(T):
            for oy in range(T):
                probe.probe_origin(L, T, ox, oy, _ip(out))
                tx, ty, q, k = out
                # reconstruct the absolute coordinates of that sub-tile site
                qx, qy = q & 1, q >> 1
                x = (ox + tx * T + qx * S + k % S) % L
                y = (oy + ty * T + qy * S + k // S) % L
                assert (x, y) == (0, 0)


@pytest.mark.parametrize("L,T", [(16, 2), (16, 4), (32, 8), (64, 16), (24, 8), (8, 8), (16, 8), (48, 16)])
@pytest.mark.parametrize("NW,B,NWT", [(1, 2, 1), (2, 2, 2), (2, 3, 1), (3, 4, 1), (4, 3, 2), (4, 2, 4), (8, 4, 4)])
def test_window_addresses_in_bounds_and_exact(probe, L, T, NW, B, NWT):
    """Every word the sweep kernels stage or write back, for every tiling
    origin, sub-tile set, tile and lane-word group, is inside the lattice and
    is the intended site's word (including the periodic wraps)."""
    probe.probe_window_check.argtypes = [ctypes.c_int] * 5 + [ctypes.POINTER(ctypes.c_longlong)]
    probe.probe_window_check.restype = ctypes.c_longlong
    n = ctypes.c_longlong()
    bad = probe.probe_window_check(L, T, NW, B, NWT, ctypes.byref(n))
    assert bad == 0 and n.value > 0


# --- (+1) tilings (section III.C) --------------------------------------------

@pytest.mark.parametrize("L,T", [(64, 6), (64, 10), (9605, 6), (9605, 10), (9605, 8), (3, 2), (37, 5),
                                 (50, 8), (27, 3), (256, 8), (130, 13), (61, 30)])
def test_general_halves_match_oracle(probe, L, T):
    """The device helper's tile halves equal the oracle's (independent code)."""
    probe.probe_gen_half.argtypes = [ctypes.c_int] * 4 + [ctypes.POINTER(ctypes.c_int)]
    probe.probe_gen_valid.restype = ctypes.c_int
    probe.probe_gen_period.restype = ctypes.c_int
    assert probe.probe_gen_valid(L, T) == 1
    assert probe.probe_gen_period(L, T) == (T if L % T == 0 else L)
    out = np.zeros(2, dtype=np.int32)
    for c in range(L // T):
        for half in (0, 1):
            probe.probe_gen_half(L, T, c, half, _ip(out))
            assert tuple(int(v) for v in out) == O.axis_half(L, T, c, half), (c, half)


def test_general_rejects_impossible_axes(probe):
    probe.probe_gen_valid.restype = ctypes.c_int
    assert probe.probe_gen_valid(10, 7) == 0   # three extra sites for one tile
    assert probe.probe_gen_valid(10, 1) == 0   # halves need a site
    assert probe.probe_gen_valid(5, 6) == 0    # no tile fits
    assert probe.probe_gen_valid(8, 3) == 1    # 3 + 1, 3 + 1


def test_general_division_exhaustive(probe):
    probe.probe_gen_div_check.restype = ctypes.c_longlong
    assert probe.probe_gen_div_check() == 0


def test_general_control_period_matches_oracle(probe):
    """The device control draw over one period of a (+1) pattern (L for an
    axis T does not divide, T otherwise) equals the oracle's."""
    out = np.zeros(6, dtype=np.int32)
    probe.probe_control.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int)]
    for (L, Tx, Ty) in [(64, 6, 10), (9605, 6, 10), (64, 8, 8)]:
        p = O.Params(L=L, N=1, Tx=Tx, Ty=Ty, seed=77, tiling=1)
        px = Tx if L % Tx == 0 else L
        py = Ty if L % Ty == 0 else L
        for t in range(50):
            ox, oy, perm = O.control(p, t)
            # probe_control takes one edge for both axes: compare each axis
            probe.probe_control(77, t, px, 0, _ip(out))
            assert int(out[0]) == ox and tuple(int(v) for v in out[2:]) == perm
            probe.probe_control(77, t, py, 0, _ip(out))
            assert int(out[1]) == oy


@pytest.mark.parametrize("L,Tx,Ty,NW,B,NWT", [
    (64, 6, 10, 2, 2, 2), (37, 4, 5, 1, 3, 1), (27, 3, 9, 3, 4, 1), (13, 2, 2, 2, 2, 1), (16, 8, 4, 2, 2, 2),
    (23, 7, 3, 2, 3, 2),
])
def test_general_window_addresses_exhaustive(probe, L, Tx, Ty, NW, B, NWT):
    """Every word the general phase kernel stages or writes back, for every
    origin of one period, set, tile and lane-word group, is inside the lattice
    and is the intended site's word; each sweep's sub-tiles cover every site
    once; the located origin slot is site (0,0)."""
    probe.probe_gen_window_check.argtypes = [ctypes.c_int] * 6 + [ctypes.POINTER(ctypes.c_longlong)]
    probe.probe_gen_window_check.restype = ctypes.c_longlong
    n = ctypes.c_longlong()
    bad = probe.probe_gen_window_check(L, Tx, Ty, NW, B, NWT, ctypes.byref(n))
    assert bad == 0 and n.value > 0


@pytest.mark.parametrize("L,Tx,Ty,NWP,wbytes,n", [
    (9605, 6, 10, 1, 16, 96), (9605, 6, 10, 1, 16, 128), (64, 6, 10, 2, 8, 64), (37, 4, 5, 3, 12, 32),
    (50, 8, 8, 2, 16, 256), (27, 3, 9, 1, 16, 64), (13, 2, 2, 32, 24, 96), (61, 30, 30, 2, 16, 32),
    (256, 8, 8, 1, 16, 192), (9, 2, 3, 1, 16, 32),
])
def test_general_launch_plan_covers_every_tile_once(probe, L, Tx, Ty, NWP, wbytes, n):
    """The general kernel's blocks (narrow, then wide with fewer threads)
    take every tile and lane-word group once, and every window fits the
    block's shared memory at its thread's slot stride."""
    probe.probe_gen_plan_check.argtypes = [ctypes.c_int] * 6 + [ctypes.POINTER(ctypes.c_longlong)]
    probe.probe_gen_plan_check.restype = ctypes.c_longlong
    out = (ctypes.c_longlong * 3)()
    assert probe.probe_gen_plan_check(L, Tx, Ty, NWP, wbytes, n, out) == 0
    assert out[0] > 0 and out[1] % 8 == 0 and out[2] <= 227 * 1024


def test_automatic_tiles_per_lane(probe):
    """The persistent engine's automatic work-item size (execution geometry):
    the choices at the lattice sizes it was measured on, and the rule's
    invariants over a grid of shapes."""
    f = probe.probe_auto_tpl
    # regular 8 x 8 tiles: L / 8 tile rows of L / 8 tiles
    for L, nwt, want in [(1024, 1, 2), (2048, 1, 2), (4096, 1, 2), (4096, 2, 2), (8192, 1, 8), (8192, 2, 4),
                         (16384, 1, 16), (32768, 1, 16), (32768, 2, 4), (32768, 4, 4)]:
        assert f(1, nwt, L // 8, L // 8) == want, (L, nwt)
    assert f(1, 2, 9605 // 10, 9605 // 6) == 4  # 6(+1) x 10(+1) at L = 9605: 960 rows of 1600 tiles
    assert [f(nwp, 1, 512, 512) for nwp in (2, 3, 4, 5, 32)] == [4, 6, 8, 8, 8]
    for nwt in (1, 2, 4):
        cap = 16 if nwt == 1 else 4
        for rows in (8, 64, 500, 1024, 4096, 8192):
            for nT in (8, 100, 512, 1600, 4096, 8192):
                t = f(1, nwt, rows, nT)
                items = lambda tpl: rows * -(-nT // (32 * tpl))
                assert t in (2, 4, 8, 16) and t <= cap
                assert t == 2 or items(t) >= 2 * 152 * 12
                assert t == cap or items(2 * t) < 2 * 152 * 12

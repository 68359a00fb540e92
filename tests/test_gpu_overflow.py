"""Exact sums beyond int64 (Eq. 2 numerators at large heights).

A job is snapshotted, every surface's absolute height of site (0,0) is
raised by D = 2^27 in the snapshot (a multiple of 2^B, so the coded residues
stay consistent and every height of the surface rises by D), and the job is
restored and advanced further.  Then sum h^2 ~ L^2 D^2 = 2^66 no longer fits
int64 while sum h^4 ~ 2^120 still fits 128 bits.  Expected values are the
oracle's heights at the same time plus D, summed exactly:

* rsos_width returns RSOS_EOVERFLOW, sum h exact, sum h^2 = INT64_MIN, and W^2
  equal to the oracle's to double rounding (it is shift invariant);
* the series read back (rsos_read_series) behaves the same;
* rsos_moments and rsos_width_noalloc give the exact 128-bit sums;
* every height of sampled lanes equals the oracle's plus D.
"""
import ctypes
import struct

import numpy as np
import pytest

import oracle as O
import paper_1605_02620_gb300 as R

pytestmark = pytest.mark.gpu

D = 1 << 27


def h00_slice(snap: bytes):
    """Byte range of the h(0,0) array (int64 per padded surface) inside a
    snapshot: header, schedule times, series times, series flags (padded to
    8), coded lattice (padded to 8), then h00."""
    header_bytes, = struct.unpack_from("<I", snap, 12)
    n_series, n_sched = struct.unpack_from("<ii", snap, header_bytes - 36)
    lattice_bytes, h00_bytes, _ = struct.unpack_from("<QQQ", snap, header_bytes - 24)
    pad8 = lambda v: (v + 7) // 8 * 8  # noqa: E731
    off = header_bytes + 8 * n_sched + 8 * n_series + pad8(n_series) + pad8(lattice_bytes)
    return off, off + h00_bytes


def to128(lo, hi):
    return (int(hi) << 64) + (int(lo) & 0xFFFFFFFFFFFFFFFF)


@pytest.mark.parametrize("L,N,S,tiling,tile", [(64, 1, 64, 0, 8), (128, 2, 96, 0, 8), (64, 1, 64, 1, (6, 10))])
def test_sums_beyond_int64_stay_exact(L, N, S, tiling, tile):
    import torch
    t1, t2 = 20, 27
    p = R.rsos_params(L=L, N=N, surfaces=S, tile=tile, seed=5, series_capacity=8, tiling=tiling)
    h = R.rsos_init(p)
    R.rsos_sweep(h, t1)
    snap = bytearray(R.rsos_snapshot(h))
    R.rsos_free(h)
    a, b = h00_slice(bytes(snap))
    h00 = np.frombuffer(bytes(snap[a:b]), dtype=np.int64).copy()
    assert len(h00) >= S
    snap[a:b] = (h00 + D).tobytes()

    nbytes = R.rsos_required_bytes(p)
    buf = torch.zeros(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = (buf.data_ptr() + 255) // 256 * 256
    h = R.rsos_restore(bytes(snap), dev_buf=base, dev_bytes=nbytes)
    try:
        R.rsos_schedule(h, [t2])
        R.rsos_sweep(h, t2 - t1)
        Tx, Ty = (tile, tile) if not isinstance(tile, tuple) else tile
        f = O.flat(L, S)
        O.sweeps(O.Params(L=L, N=N, Tx=Tx, Ty=Ty, seed=5, tiling=tiling), f, list(range(S)), 0, t2)
        f += D
        o1, o2 = O.sums(f)
        ops = O.power_sums(f)
        assert all(v >= 1 << 63 for v in o2) and all(v < 1 << 127 for r in ops for v in r)

        # rsos_width: status RSOS_EOVERFLOW, sum h exact, sum h^2 flagged, W^2 exact
        s1 = np.zeros(S, dtype=np.int64)
        s2 = np.zeros(S, dtype=np.int64)
        w2 = np.zeros(S, dtype=np.float64)
        t = ctypes.c_int64()
        P = lambda a, c: a.ctypes.data_as(ctypes.POINTER(c))  # noqa: E731
        rc = R._load().rsos_width(h, P(s1, ctypes.c_int64), P(s2, ctypes.c_int64), P(w2, ctypes.c_double),
                                  ctypes.byref(t), None)
        assert rc == R.RSOS_EOVERFLOW and t.value == t2
        for j in range(S):
            assert int(s1[j]) == o1[j]
            assert int(s2[j]) == -(1 << 63)
            w = O.width2(o1[j], o2[j], L)
            assert abs(w2[j] - w) <= 1e-9 * max(1.0, w), (j, w2[j], w)

        # the scheduled measurement at t2, read back through the series
        ts, r1, r2, rw = R.rsos_read_series(h, S, 8, allow_overflow=True)
        assert list(ts) == [t2]
        assert [int(v) for v in r1[0]] == o1 and all(int(v) == -(1 << 63) for v in r2[0])
        assert np.allclose(rw[0], w2, rtol=1e-12, atol=0)

        # 128-bit exports: moments and the allocation-free measurement
        tm, sums = R.rsos_moments(h, S)
        assert tm == t2
        for j in range(S):
            assert [int(v) for v in sums[j]] == ops[j], j
        out = torch.full((S * 4,), -1, dtype=torch.int64, device="cuda")
        B = 2 if N <= 1 else (3 if N <= 3 else 4)
        NW = (S + 31) // 32
        rows = L * Tx * ((L + Tx - 1) // Tx) if tiling else L * L
        h00_off = (B * rows * NW * 4 + 255) // 256 * 256
        R.rsos_width_noalloc(p, base, base + h00_off, out.data_ptr())
        torch.cuda.synchronize()
        v = out.cpu().numpy().reshape(S, 4)
        assert [to128(x, y) for x, y in v[:, 0:2]] == o1
        assert [to128(x, y) for x, y in v[:, 2:4]] == o2

        for j in (0, S - 1):
            assert np.array_equal(R.rsos_heights(h, j, L), f[j])
    finally:
        R.rsos_free(h)

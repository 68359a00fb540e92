"""Brute-force check of the persistent engine's work order and dependency
rules (product code compiled for the host), on small lattices and random
tilings:

* tickets enumerate every item (t, p, r, c) of every sweep exactly once;
* every dependency refers to items with smaller tickets, so the lowest
  unfinished ticket can always run (no deadlock with all blocks resident);
* per tile row the completion counter is monotone: sweep t+1's items of a
  row depend transitively on all of sweep t's items of that row;
* every pair of activations that touch a common site, at least one of them
  writing it, is ordered by a dependency path in sequential (t, p) order;
  activations of one phase never conflict.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1605_02620_gb300", "csrc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("sched") / "probe.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-I", CSRC,
                           os.path.join(HERE, "host", "logic_probe.cpp"), "-o", out])
    lib = ctypes.CDLL(out)
    ip = ctypes.POINTER(ctypes.c_int)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.probe_order_table.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p]
    lib.probe_order_entry.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, ip]
    lib.probe_item.argtypes = [ip, ctypes.c_uint64, ctypes.c_uint32, ip]
    lib.probe_deps.argtypes = [ip, ip, ctypes.POINTER(ctypes.c_int64)]
    lib.probe_gen_item.argtypes = [ip, ctypes.c_uint64, ctypes.c_uint32, ip]
    lib.probe_gen_deps.argtypes = [ip, ip, ctypes.POINTER(ctypes.c_int64)]
    return lib


@pytest.mark.parametrize("nT,K,D", [
    (1, 1, 2), (2, 3, 2), (3, 1, 2), (5, 2, 3), (8, 4, 2), (8, 1, 9), (12, 3, 4), (12, 2, 5),
    (31, 3, 7), (64, 8, 21), (64, 2, 40), (512, 8, 91), (512, 8, 170), (512, 4, 300),
    # the automatic geometries of large lattices (8 x 8 tiles, 1824 workers):
    # L = 8192 with 8 (32-bit) and 4 (64-bit) tiles per lane, L = 16384 and
    # 32768 with 16 (32-bit), L = 32768 with 4 (64-bit)
    (1024, 4, 341), (1024, 8, 171), (2048, 4, 342), (4096, 8, 171), (4096, 32, 42),
])
def test_order_entry_matches_table(probe, nT, K, D):
    """The device computes a ticket's (phase, visit row, chunk) arithmetically;
    it must enumerate exactly the slot-ordered table, including phase lags
    above nT/3 where the phase fronts overlap differently."""
    table = np.zeros(4 * nT * K, dtype=np.uint32)
    n = probe.probe_order_table(nT, K, D, table.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    assert n == 4 * nT * K
    out = np.zeros(3, dtype=np.int32)
    for e in range(n):
        probe.probe_order_entry(nT, K, D, e, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        v = int(table[e])
        assert (int(out[0]), int(out[1]), int(out[2])) == (v & 3, (v >> 2) & 0x3FFFF, v >> 20), e


def _footprint(L, T, ox, oy, q, ty, txs):
    """Sites written (sub-tile) and touched (sub-tile + halo) by an item."""
    S = T // 2
    qx, qy = q & 1, q >> 1
    wr, rd = set(), set()
    for tx in txs:
        for ky in range(-1, S + 1):
            for kx in range(-1, S + 1):
                inside = 0 <= kx < S and 0 <= ky < S
                edge = (kx in (-1, S)) != (ky in (-1, S))
                if not inside and not edge:
                    continue
                x = (ox + tx * T + qx * S + kx) % L
                y = (oy + ty * T + qy * S + ky) % L
                rd.add((x, y))
                if inside:
                    wr.add((x, y))
    return wr, rd


@pytest.mark.parametrize("L,T,CW,D,seed,order", [
    (32, 8, 2, 2, 1, 0), (32, 8, 4, 3, 2, 0), (24, 8, 1, 2, 3, 0), (16, 4, 3, 2, 4, 0),
    (16, 2, 4, 2, 5, 0), (8, 2, 8, 3, 6, 1), (8, 8, 1, 2, 7, 0), (16, 8, 2, 2, 8, 0),
])
def test_schedule_is_sound(probe, L, T, CW, D, seed, order):
    nT = L // T
    K = -(-nT // CW)
    n_sweeps = 6
    g8 = np.array([L, T, K, D, order, seed, 0, 0], dtype=np.int32)
    gp = g8.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    table = np.zeros(4 * nT * K, dtype=np.uint32)
    n = probe.probe_order_table(nT, K, D, table.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    assert n == 4 * nT * K
    items, ticket_of = [], {}
    out = np.zeros(4, dtype=np.int32)
    for tk in range(n_sweeps * n):
        probe.probe_item(gp, tk, 0, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        it = tuple(int(v) for v in out)
        assert it not in ticket_of
        ticket_of[it] = tk
        items.append(it)
    assert set(ticket_of) == {(t, p, r, c) for t in range(n_sweeps) for p in range(4)
                              for r in range(nT) for c in range(K)}
    # direct dependencies as item sets
    deps = {}
    buf = np.zeros(12, dtype=np.int64)
    for it in items:
        a = np.array(it, dtype=np.int32)
        k = probe.probe_deps(gp, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                             buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        ds = set()
        for m in range(k):
            p2, r2, target = int(buf[3 * m]), int(buf[3 * m + 1]), int(buf[3 * m + 2])
            assert target % K == 0
            td = target // K - 1
            assert td <= it[0]
            for t2 in range(td + 1):
                for c2 in range(K):
                    ds.add((t2, p2, r2, c2))
        for d in ds:
            assert ticket_of[d] < ticket_of[it], (it, d)
        deps[it] = ds
    # transitive closure in ticket order
    index = {it: i for i, it in enumerate(items)}
    reach = [0] * len(items)
    for i, it in enumerate(items):
        m = 0
        for d in deps[it]:
            j = index[d]
            m |= reach[j] | (1 << j)
        reach[i] = m

    def depends(a, b):
        return bool((reach[index[a]] >> index[b]) & 1)

    # counters are monotone per row
    for (t, p, r, c) in items:
        if t + 1 < n_sweeps:
            for c2 in range(K):
                assert depends((t + 1, p, r, c), (t, p, r, c2))
    # conflicts are ordered
    p_ = O.Params(L=L, N=1, Tx=T, Ty=T, phase_order=order, seed=seed)
    foot = {}
    for (t, p, r, c) in items:
        ox, oy, perm = O.control(p_, t)
        txs = [tx for tx in range(c * CW, min(nT, (c + 1) * CW))]
        foot[(t, p, r, c)] = _footprint(L, T, ox, oy, perm[p], r, txs)
    seq = sorted(items, key=lambda it: (it[0], it[1]))
    for i, a in enumerate(seq):
        wa, ra = foot[a]
        for b in seq[i + 1:]:
            wb, rb = foot[b]
            if not (wa & rb or ra & wb):
                continue
            assert (a[0], a[1]) != (b[0], b[1]), ("same-phase conflict", a, b)
            assert depends(b, a), (b, "must depend on", a)


def _gen_footprint(L, Tx, Ty, ox, oy, q, ty, txs):
    """Sites written (sub-tile) and touched (sub-tile + halo) by an item of a
    (+1) tiling, from the oracle's own tiling geometry (axis_half)."""
    qx, qy = q & 1, q >> 1
    v0, sh = O.axis_half(L, Ty, ty, qy)
    wr, rd = set(), set()
    for tx in txs:
        u0, sw = O.axis_half(L, Tx, tx, qx)
        for ky in range(-1, sh + 1):
            for kx in range(-1, sw + 1):
                inside = 0 <= kx < sw and 0 <= ky < sh
                edge = (kx in (-1, sw)) != (ky in (-1, sh))
                if not inside and not edge:
                    continue
                site = ((ox + u0 + kx) % L, (oy + v0 + ky) % L)
                rd.add(site)
                if inside:
                    wr.add(site)
    return wr, rd


@pytest.mark.parametrize("L,Tx,Ty,CW,D,seed,order", [
    (13, 3, 4, 2, 2, 1, 0), (20, 6, 4, 1, 2, 2, 0), (17, 4, 2, 2, 3, 3, 0), (14, 2, 3, 3, 2, 4, 1),
    (22, 6, 10, 1, 2, 5, 0), (16, 8, 8, 1, 2, 6, 0), (11, 2, 2, 2, 2, 7, 0), (25, 4, 6, 2, 3, 8, 0),
])
def test_general_schedule_is_sound(probe, L, Tx, Ty, CW, D, seed, order):
    """The (+1)-tiling schedule: every item once, dependencies earlier in
    ticket order, per-row completion counters monotone, and every pair of
    conflicting activations (a common site, one of them writing it) ordered
    by a dependency path in sequential (t, p) order.  Footprints come from
    the oracle's tiling geometry and control draw, not from the product."""
    nx, ny = L // Tx, L // Ty
    K = -(-nx // CW)
    n_sweeps = 6
    g8 = np.array([L, Tx, Ty, K, D, order, seed, 0], dtype=np.int32)
    gp = g8.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    n = 4 * ny * K
    items, ticket_of = [], {}
    out = np.zeros(4, dtype=np.int32)
    for tk in range(n_sweeps * n):
        probe.probe_gen_item(gp, tk, 0, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        it = tuple(int(v) for v in out)
        assert it not in ticket_of
        ticket_of[it] = tk
        items.append(it)
    assert set(ticket_of) == {(t, p, r, c) for t in range(n_sweeps) for p in range(4)
                              for r in range(ny) for c in range(K)}
    deps = {}
    buf = np.zeros(12, dtype=np.int64)
    for it in items:
        a = np.array(it, dtype=np.int32)
        k = probe.probe_gen_deps(gp, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 buf.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        ds = set()
        for m in range(k):
            p2, r2, target = int(buf[3 * m]), int(buf[3 * m + 1]), int(buf[3 * m + 2])
            assert target % K == 0 and 0 <= r2 < ny
            td = target // K - 1
            assert td <= it[0]
            for t2 in range(td + 1):
                for c2 in range(K):
                    ds.add((t2, p2, r2, c2))
        for d in ds:
            assert ticket_of[d] < ticket_of[it], (it, d)
        deps[it] = ds
    index = {it: i for i, it in enumerate(items)}
    reach = [0] * len(items)
    for i, it in enumerate(items):
        m = 0
        for d in deps[it]:
            j = index[d]
            m |= reach[j] | (1 << j)
        reach[i] = m

    def depends(a, b):
        return bool((reach[index[a]] >> index[b]) & 1)

    for (t, p, r, c) in items:
        if t + 1 < n_sweeps:
            for c2 in range(K):
                assert depends((t + 1, p, r, c), (t, p, r, c2))
    p_ = O.Params(L=L, N=1, Tx=Tx, Ty=Ty, phase_order=order, seed=seed, tiling=1)
    foot = {}
    for (t, p, r, c) in items:
        ox, oy, perm = O.control(p_, t)
        txs = [tx for tx in range(c * CW, min(nx, (c + 1) * CW))]
        foot[(t, p, r, c)] = _gen_footprint(L, Tx, Ty, ox, oy, perm[p], r, txs)
    seq = sorted(items, key=lambda it: (it[0], it[1]))
    for i, a in enumerate(seq):
        wa, ra = foot[a]
        for b in seq[i + 1:]:
            wb, rb = foot[b]
            if not (wa & rb or ra & wb):
                continue
            assert (a[0], a[1]) != (b[0], b[1]), ("same-phase conflict", a, b)
            assert depends(b, a), (b, "must depend on", a)

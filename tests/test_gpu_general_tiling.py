"""(+1) tilings of the decomposition check (section III.C: 6(+1) x 10(+1)
domains) on the GPU against the oracle, bit for bit: sums, W^2 and heights
of every lane.  Plus: with T even and dividing L the general engine is the
regular tiling (bit-identical to the regular engines, up to L = 4096); the
paper's largest lattice, L = 9605, against the oracle on sampled lanes; a
checkpoint round trip; exact power sums; batches, rsos_advance and the
no-allocation width on (+1)-tiling jobs."""
import numpy as np
import pytest

import oracle as O
import paper_1605_02620_gb300 as R
from rsos_testlib import assert_parity, gpu_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,N,S,T,order,t_end", [
    (64, 1, 64, (6, 10), 0, 30),    # the paper's 6(+1) x 10(+1) at its smallest L
    (64, 3, 32, (6, 10), 0, 25),    # 3 planes, one 32-bit lane word
    (37, 2, 96, (4, 5), 0, 30),     # three lane words (32-bit), ragged tiles on both axes
    (50, 1, 128, (8, 8), 1, 30),    # 8(+1), fixed phase order, 64-bit words in pairs
    (27, 7, 64, (3, 9), 0, 20),     # odd regular tiles (T divides L): halves 1 + 2, 4 + 5
    (13, 2, 2048, (2, 2), 0, 12),   # 64 lane words; halves of 1 and 2 sites
    (9, 1, 64, (2, 3), 0, 40),      # one axis irregular, the other regular and odd
    (61, 4, 64, (30, 30), 0, 8),    # the widest tiles: halves of 15 and 16 sites
])
def test_general_tiling_matches_oracle(L, N, S, T, order, t_end):
    times = sorted({0, 1, 3, t_end // 2, t_end})
    assert_parity(L, N, S, T, seed=41 + L + N, order=order, times=times, t_end=t_end, tiling=1)


@pytest.mark.parametrize("L,N,S,T,order,t_end", [
    (64, 1, 64, (6, 10), 0, 30),
    (64, 3, 32, (6, 10), 0, 25),
    (37, 2, 96, (4, 5), 0, 30),
    (50, 1, 128, (8, 8), 1, 30),
    (27, 7, 64, (3, 9), 0, 20),
    (13, 2, 2048, (2, 2), 0, 12),
    (9, 1, 64, (2, 3), 0, 40),
    (130, 1, 64, (6, 10), 0, 24),   # 13 tile rows
])
def test_persistent_engine_on_general_tilings_matches_oracle(L, N, S, T, order, t_end):
    """The persistent dataflow engine on (+1) tilings (its own work order:
    tile rows T or T + 1 high, the origin anywhere in the pattern's period)
    against the oracle, bit for bit, on the tilings above, down to one or
    two tile rows per axis."""
    times = sorted({0, 1, 3, t_end // 2, t_end})
    assert_parity(L, N, S, T, seed=41 + L + N, order=order, times=times, t_end=t_end, tiling=1, engine=2)


def test_persistent_and_phase_engines_agree_at_L9605():
    kw = dict(L=9605, N=1, S=64, T=(6, 10), seed=21, times=[0, 1, 5, 12], t_end=12, height_lanes=[0, 63],
              tiling=1)
    a = gpu_run(engine=1, **kw)
    b = gpu_run(engine=2, **kw)
    assert (a[1] == b[1]).all() and (a[2] == b[2]).all()
    for j in (0, 63):
        assert np.array_equal(a[4][j], b[4][j]), j


def test_persistent_engine_wait_timeout_on_general_tiling():
    p = R.rsos_params(L=130, N=1, surfaces=64, tile=(6, 10), seed=2, engine=2, tiling=1, series_capacity=4)
    h = R.rsos_init(p)
    try:
        R.rsos_sweep(h, 3)
        s1, s2, _, _ = R.rsos_width(h, 64)
        assert R.rsos_selftest_timeout(h, 20_000_000) == R.RSOS_ETIMEOUT
        # the lattice is untouched and the handle keeps working
        t1, t2, _, _ = R.rsos_width(h, 64)
        assert (s1 == t1).all() and (s2 == t2).all()
        R.rsos_sweep(h, 2)
        assert R.rsos_time(h) == 5
    finally:
        R.rsos_free(h)


@pytest.mark.parametrize("L,N,S,T", [(256, 1, 64, 8), (128, 2, 32, 4), (64, 5, 64, 16)])
def test_divisible_tiles_equal_the_regular_engines(L, N, S, T):
    kw = dict(L=L, N=N, S=S, T=T, seed=7, times=[0, 3, 11], t_end=11, height_lanes=[0, S - 1])
    g = gpu_run(tiling=1, **kw)
    for engine in (1, 2) if L // T >= 8 else (1,):
        r = gpu_run(engine=engine, **kw)
        assert (g[1] == r[1]).all() and (g[2] == r[2]).all(), engine
        for j in (0, S - 1):
            assert np.array_equal(g[4][j], r[4][j]), (engine, j)


def test_divisible_tiles_equal_the_persistent_engine_full_size():
    kw = dict(L=4096, N=1, S=64, T=8, seed=9, times=[0, 1, 7, 20], t_end=20, height_lanes=[0, 40])
    g = gpu_run(tiling=1, **kw)
    r = gpu_run(engine=2, **kw)
    assert (g[1] == r[1]).all() and (g[2] == r[2]).all()
    for j in (0, 40):
        assert np.array_equal(g[4][j], r[4][j])


def test_L9605_against_oracle_on_sampled_lanes():
    """L = 9605 (the paper's largest lattice; not a multiple of 6 or 10),
    6(+1) x 10(+1), 64 surfaces: two lanes' sums and every height after 2
    sweeps equal the oracle's."""
    L, t_end, lanes = 9605, 2, [0, 45]
    gts, g1, g2, gw, gh = gpu_run(L, 1, 64, (6, 10), seed=5, times=[0, 1, 2], t_end=t_end, height_lanes=lanes,
                                  tiling=1)
    p = O.Params(L=L, N=1, Tx=6, Ty=10, seed=5, tiling=1)
    ts, o1, o2, oh = O.run_series(p, lanes, [0, 1, 2], threads=2)
    assert list(gts) == ts
    for m in range(len(ts)):
        for c, j in enumerate(lanes):
            assert int(g1[m, j]) == int(o1[m][c]) and int(g2[m, j]) == int(o2[m][c]), (ts[m], j)
    for c, j in enumerate(lanes):
        assert np.array_equal(gh[j], oh[c]), j


def test_L9605_longer_run_properties():
    """After 40 sweeps at L = 9605: every neighbour difference of the read-back
    heights is within N (Eq. 6, periodic), and their exact sums are the
    measured ones."""
    L, N, S = 9605, 2, 32
    gts, g1, g2, gw, gh = gpu_run(L, N, S, (6, 10), seed=8, times=[40], t_end=40, height_lanes=[0, 31],
                                  tiling=1)
    for j in (0, 31):
        h = gh[j].astype(np.int64)
        assert np.abs(h - np.roll(h, 1, axis=0)).max() <= N
        assert np.abs(h - np.roll(h, 1, axis=1)).max() <= N
        assert int(h.sum()) == int(g1[0, j])
        assert int((h * h).sum()) == int(g2[0, j])
        assert h.sum() > 0.3 * 40 * L * L  # it grew


def test_checkpoint_round_trip():
    times = [0, 2, 5, 9]
    p = R.rsos_params(L=64, N=1, surfaces=64, tile=(6, 10), seed=3, series_capacity=8, tiling=1)
    a = R.rsos_init(p)
    R.rsos_schedule(a, times)
    R.rsos_sweep(a, 9)
    ref = R.rsos_read_series(a, 64, 8)
    ref_h = R.rsos_heights(a, 17, 64)
    R.rsos_free(a)
    b = R.rsos_init(p)
    R.rsos_schedule(b, times)
    R.rsos_sweep(b, 4)
    snap = R.rsos_snapshot(b)
    R.rsos_free(b)
    c = R.rsos_restore(snap)
    try:
        R.rsos_sweep(c, 5)
        got = R.rsos_read_series(c, 64, 8)
        got_h = R.rsos_heights(c, 17, 64)
    finally:
        R.rsos_free(c)
    assert list(got[0]) == list(ref[0]) == times
    assert (got[1] == ref[1]).all() and (got[2] == ref[2]).all()
    assert np.array_equal(got_h, ref_h)


def test_power_sums_match_oracle():
    """Sum h^3, sum h^4 (section III.C moments) on a (+1) tiling, exactly."""
    L, N, S, t_end, times = 64, 2, 64, 15, [0, 4, 15]
    p = R.rsos_params(L=L, N=N, surfaces=S, tile=(6, 10), seed=13, series_capacity=8, tiling=1)
    h = R.rsos_init(p)
    try:
        R.rsos_set_moments(h, True)
        R.rsos_schedule(h, times)
        R.rsos_sweep(h, t_end)
        ts, sums, has = R.rsos_read_moments(h, S, 8)
    finally:
        R.rsos_free(h)
    ots, _, _, _, ops = O.run_series(O.Params(L=L, N=N, Tx=6, Ty=10, seed=13, tiling=1), list(range(S)), times,
                                     powers=True)
    assert list(ts) == ots and has.all()
    for m in range(len(ots)):
        for j in range(S):
            assert list(sums[m, j]) == ops[m][j], (ots[m], j)


def test_batch_and_advance_run_general_jobs():
    """(+1)-tiling jobs in a batch (beside regular jobs) and through
    rsos_advance give what they give alone."""
    import torch
    jobs = [(64, 1, 64, (6, 10), 1, 20), (128, 1, 64, 8, 0, 15), (37, 2, 96, (4, 5), 1, 12)]
    params = [R.rsos_params(L=L, N=N, surfaces=S, tile=T, seed=k, series_capacity=4, tiling=tl)
              for k, (L, N, S, T, tl, t) in enumerate(jobs)]
    b = R.rsos_batch_create(params, [t for (*_, t) in jobs])
    try:
        R.rsos_batch_run(b, torch.cuda.Stream())
        done = set()
        for _ in range(200000):
            rc, ids = R.rsos_batch_poll(b)
            done |= set(ids)
            if len(done) == len(jobs):
                break
        assert len(done) == len(jobs)
        got = [R.rsos_read_series(R.rsos_batch_job(b, k), jobs[k][2], 4) for k in range(len(jobs))]
    finally:
        R.rsos_batch_free(b)
    handles = [R.rsos_init(p) for p in params]
    try:
        for h, (*_, t) in zip(handles, jobs):
            R.rsos_schedule(h, [t])
        R.rsos_advance(handles, [t for (*_, t) in jobs])
        adv = [R.rsos_read_series(h, jobs[k][2], 4) for k, h in enumerate(handles)]
    finally:
        for h in handles:
            R.rsos_free(h)
    for k, (L, N, S, T, tl, t) in enumerate(jobs):
        _, a1, a2, _, _ = gpu_run(L, N, S, T, seed=k, times=[t], t_end=t, tiling=tl)
        for res in (got[k], adv[k]):
            assert list(res[0]) == [t]
            assert (res[1] == a1).all() and (res[2] == a2).all(), k


def test_noalloc_width_on_general_layout():
    """rsos_width_noalloc reads the padded class-interleaved records of a (+1)
    tiling."""
    import torch
    L, S = 64, 64
    p = R.rsos_params(L=L, N=1, surfaces=S, tile=(6, 10), seed=21, series_capacity=4, tiling=1)
    nbytes = R.rsos_required_bytes(p)
    buf = torch.zeros(nbytes + 256, dtype=torch.uint8, device="cuda")
    base = (buf.data_ptr() + 255) // 256 * 256
    # planes: L rows of 6 ceil(L / 6) 16-byte records (class-interleaved, padded)
    h00_off = (2 * L * 6 * ((L + 5) // 6) * 2 * 4 + 255) // 256 * 256
    out = torch.zeros(S * 4, dtype=torch.int64, device="cuda")
    h = R.rsos_init(p, dev_buf=base, dev_bytes=nbytes)
    try:
        R.rsos_sweep(h, 9)
        s1, s2, _, _ = R.rsos_width(h, S)
        R.rsos_width_noalloc(p, base, base + h00_off, out.data_ptr())
        torch.cuda.synchronize()
    finally:
        R.rsos_free(h)
    v = out.cpu().numpy().reshape(S, 4)
    to128 = lambda lo, hi: [(int(b) << 64) + (int(a) & 0xFFFFFFFFFFFFFFFF) for a, b in zip(lo, hi)]
    assert to128(v[:, 0], v[:, 1]) == [int(x) for x in s1]
    assert to128(v[:, 2], v[:, 3]) == [int(x) for x in s2]

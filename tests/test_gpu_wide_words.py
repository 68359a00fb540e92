"""128-lane words (rsos_params.words_per_thread = 4).  Section II groups the
realizations of one SIMT unit by 128 with one site sequence; here a thread
can hold four 32-lane words of a site as one 128-lane word.  The word width a
thread holds is execution geometry: the same job gives the oracle's sums and
heights bit for bit whether its threads hold 32, 64 or 128 lanes, with one
or several 128-lane groups per tile, on the single-job engine, through a batch
and through rsos_advance, and a wait that can never be satisfied still ends
with RSOS_ETIMEOUT."""
import numpy as np
import pytest

import paper_1605_02620_gb300 as R
from rsos_testlib import gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,N,S,t_end", [
    (64, 1, 128, 40),   # one 128-lane group per tile: whole 32-byte records
    (128, 2, 128, 25),  # 3 bit planes
    (64, 4, 256, 20),   # two groups per tile: plane-by-plane 16-byte copies
    (96, 5, 384, 12),   # three groups per tile (30 of 32 lanes busy), 4 planes
    (64, 7, 128, 12),
])
def test_wide_words_match_oracle(L, N, S, t_end):
    times = sorted({0, 1, 3, t_end // 2, t_end})
    gts, g1, g2, _, gh = gpu_run(L, N, S, 8, seed=57 + N, times=times, t_end=t_end,
                                 height_lanes=list(range(S)), engine=2, words_per_thread=4)
    ots, o1, o2, oh = oracle_run(L, N, list(range(S)), 8, seed=57 + N, times=times, t_end=t_end)
    assert list(gts) == list(ots)
    for m in range(len(ots)):
        assert [int(v) for v in g1[m]] == [int(v) for v in o1[m]], ots[m]
        assert [int(v) for v in g2[m]] == [int(v) for v in o2[m]], ots[m]
    for j in range(S):
        assert np.array_equal(gh[j], oh[j]), j


@pytest.mark.parametrize("N", [1, 2])
def test_word_width_is_invisible(N):
    kw = dict(L=256, N=N, S=128, T=8, seed=23, times=[0, 4, 11], t_end=11, height_lanes=[0, 63, 64, 127])
    base = gpu_run(engine=2, words_per_thread=4, **kw)
    for wpt, tpl in [(1, 0), (2, 0), (4, 1), (4, 3)]:
        other = gpu_run(engine=2, words_per_thread=wpt, tiles_per_lane=tpl, **kw)
        assert (base[1] == other[1]).all() and (base[2] == other[2]).all(), (wpt, tpl)
        for j in (0, 63, 64, 127):
            assert np.array_equal(base[4][j], other[4][j]), (wpt, tpl, j)


def test_wide_word_jobs_in_a_batch_and_through_advance():
    import torch
    jobs = [(64, 1, 128, 4, 20), (128, 1, 64, 0, 15), (64, 2, 256, 4, 12)]
    params = [R.rsos_params(L=L, N=N, surfaces=S, seed=k, series_capacity=4, words_per_thread=w)
              for k, (L, N, S, w, t) in enumerate(jobs)]
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
    for k, (L, N, S, w, t) in enumerate(jobs):
        _, a1, a2, _, _ = gpu_run(L, N, S, 8, seed=k, times=[t], t_end=t)  # automatic word width
        for res in (got[k], adv[k]):
            assert list(res[0]) == [t]
            assert (res[1] == a1).all() and (res[2] == a2).all(), k


def test_wide_word_wait_timeout_is_reported():
    p = R.rsos_params(L=64, N=1, surfaces=128, tile=8, seed=4, engine=2, series_capacity=8, words_per_thread=4)
    h = R.rsos_init(p)
    try:
        R.rsos_sweep(h, 3)
        assert R.rsos_selftest_timeout(h, 20_000_000) == -5  # RSOS_ETIMEOUT, 20 ms per wait
        assert R.rsos_time(h) == 3
        R.rsos_schedule(h, [9])
        R.rsos_sweep(h, 6)
        ts, s1, s2, _ = R.rsos_read_series(h, 128, 4)
    finally:
        R.rsos_free(h)
    ots, o1, o2, _ = oracle_run(64, 1, list(range(128)), 8, seed=4, times=[9], t_end=9)
    assert list(ts) == [9]
    assert [int(v) for v in s1[0]] == [int(v) for v in o1[0]]
    assert [int(v) for v in s2[0]] == [int(v) for v in o2[0]]

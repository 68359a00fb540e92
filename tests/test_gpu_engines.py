"""The persistent dataflow engine (engine 2) against the oracle and against
the one-launch-per-phase engine (engine 1): results must be bit-identical
whatever engine, block geometry or tile size runs them.  Plus the
fault-detection check: a persistent launch whose dependency waits can never be
satisfied ends with RSOS_ETIMEOUT and leaves the GPU and the handle usable."""
import numpy as np
import pytest

import paper_1605_02620_gb300 as R
from rsos_testlib import assert_parity, gpu_run, oracle_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("L,N,S,T,t_end", [
    (64, 1, 64, 8, 40), (128, 2, 64, 8, 25), (64, 4, 32, 8, 30), (32, 1, 64, 4, 40),
    (16, 3, 96, 2, 40), (64, 7, 128, 16, 10), (8, 1, 64, 8, 30), (24, 2, 32, 8, 30),
    (16, 2, 2048, 8, 12),  # 64 lane words: uint64 words with 3 planes, 32 threads per tile
])
def test_persistent_engine_matches_oracle(L, N, S, T, t_end):
    times = sorted({0, 1, 3, t_end // 2, t_end})
    gts, g1, g2, gw, gh = gpu_run(L, N, S, T, seed=31 + L + N, times=times, t_end=t_end,
                                  height_lanes=list(range(S)), engine=2)
    ots, o1, o2, oh = oracle_run(L, N, list(range(S)), T, seed=31 + L + N, times=times, t_end=t_end)
    assert list(gts) == list(ots)
    for m in range(len(ots)):
        assert [int(v) for v in g1[m]] == [int(v) for v in o1[m]]
        assert [int(v) for v in g2[m]] == [int(v) for v in o2[m]]
    for j in range(S):
        assert np.array_equal(gh[j], oh[j]), j


def test_engines_bit_identical_full_size():
    kw = dict(L=4096, N=1, S=64, T=8, seed=9, times=[0, 1, 7, 20], t_end=20, height_lanes=[0, 40])
    a = gpu_run(engine=1, **kw)
    b = gpu_run(engine=2, **kw)
    assert (a[1] == b[1]).all() and (a[2] == b[2]).all()
    for j in (0, 40):
        assert np.array_equal(a[4][j], b[4][j])


@pytest.mark.parametrize("N", [1, 2])
def test_execution_geometry_is_invisible(N, monkeypatch):
    """Word width per thread, tiles per lane and phase lag change only how the
    work is scheduled: sums and heights must not move."""
    kw = dict(L=256, N=N, S=64, T=8, seed=17, times=[0, 2, 9], t_end=9, height_lanes=[0, 33, 63], engine=2)
    base = gpu_run(**kw)
    for env in ({"RSOS_WORDS_PER_THREAD": "1"}, {"RSOS_TILES_PER_LANE": "1"}, {"RSOS_TILES_PER_LANE": "3"},
                {"RSOS_PHASE_LAG": "2"}, {"RSOS_PHASE_LAG": "40"}):
        with monkeypatch.context() as m:
            for k, v in env.items():
                m.setenv(k, v)
            other = gpu_run(**kw)
        assert (base[1] == other[1]).all() and (base[2] == other[2]).all(), env
        for j in (0, 33, 63):
            assert np.array_equal(base[4][j], other[4][j]), (env, j)


def test_timeout_is_reported_and_gpu_stays_usable():
    p = R.rsos_params(L=64, N=1, surfaces=64, tile=8, seed=4, engine=2, series_capacity=8)
    h = R.rsos_init(p)
    try:
        R.rsos_sweep(h, 3)
        rc = R.rsos_selftest_timeout(h, 20_000_000)  # 20 ms per wait
        assert rc == -5  # RSOS_ETIMEOUT
        assert R.rsos_time(h) == 3
        # still usable and still exact
        R.rsos_schedule(h, [10])
        R.rsos_sweep(h, 7)
        ts, s1, s2, _ = R.rsos_read_series(h, 64, 4)
        assert list(ts) == [10]
    finally:
        R.rsos_free(h)
    ots, o1, o2, _ = oracle_run(64, 1, list(range(64)), 8, seed=4, times=[10], t_end=10)
    assert [int(v) for v in s1[0]] == [int(v) for v in o1[0]]
    assert [int(v) for v in s2[0]] == [int(v) for v in o2[0]]

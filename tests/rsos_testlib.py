"""Helpers shared by the GPU parity tests: run a job through the C ABI and the
same job through the oracle."""
import numpy as np

import oracle as O
import paper_1605_02620_gb300 as R


def _edges(T):
    return (T, T) if not isinstance(T, (tuple, list)) else tuple(T)


def gpu_run(L, N, S, T=8, seed=0, order=0, times=(), t_end=0, height_lanes=(), engine=0, stream=None, tiling=0,
            words_per_thread=0, tiles_per_lane=0):
    """Run a job from the flat start to t_end through the C ABI, measuring at
    ``times``.  T is a square edge or (Tx, Ty); tiling 1 selects the (+1)
    tilings; words_per_thread / tiles_per_lane set the persistent engine's
    execution geometry (0: automatic).  Returns (times, sum_h[n, S],
    sum_h2[n, S], w2[n, S], heights)."""
    times = sorted(set(int(v) for v in times))
    p = R.rsos_params(L=L, N=N, surfaces=S, tile=_edges(T), phase_order=order, seed=seed, engine=engine,
                      series_capacity=max(len(times) + 1, 4), tiling=tiling, words_per_thread=words_per_thread,
                      tiles_per_lane=tiles_per_lane)
    h = R.rsos_init(p, stream=stream)
    try:
        R.rsos_schedule(h, times)
        R.rsos_sweep(h, t_end, stream=stream)
        ts, s1, s2, w2 = R.rsos_read_series(h, S, len(times) + 1, stream=stream)
        heights = {j: R.rsos_heights(h, j, L, stream=stream) for j in height_lanes}
        assert R.rsos_time(h) == t_end
    finally:
        R.rsos_free(h)
    return ts, s1, s2, w2, heights


def oracle_run(L, N, lanes, T=8, seed=0, order=0, times=(), t_end=0, threads=None, tiling=0):
    """The same job on the oracle for the given lanes.  Returns
    (times, sum_h[n, lanes], sum_h2[n, lanes], final heights[lanes, L, L])."""
    times = sorted(set(int(v) for v in times) | {t_end})
    Tx, Ty = _edges(T)
    p = O.Params(L=L, N=N, Tx=Tx, Ty=Ty, phase_order=order, seed=seed, tiling=tiling)
    ts, s1, s2, h = O.run_series(p, lanes, times, threads=threads)
    return ts, np.array(s1, dtype=object), np.array(s2, dtype=object), h


def assert_parity(L, N, S, T=8, seed=0, order=0, times=(), t_end=0, lanes=None, height_lanes=None, threads=None,
                  tiling=0, engine=0):
    lanes = list(range(S)) if lanes is None else list(lanes)
    height_lanes = lanes if height_lanes is None else list(height_lanes)
    times = sorted(set(int(v) for v in times) | {t_end})
    gts, g1, g2, gw, gh = gpu_run(L, N, S, T, seed, order, times, t_end, height_lanes, engine=engine, tiling=tiling)
    ots, o1, o2, oh = oracle_run(L, N, lanes, T, seed, order, times, t_end, threads, tiling=tiling)
    assert list(gts) == list(ots)
    for m in range(len(ots)):
        for c, j in enumerate(lanes):
            assert int(g1[m, j]) == int(o1[m, c]), (ots[m], j, "sum h")
            assert int(g2[m, j]) == int(o2[m, c]), (ots[m], j, "sum h^2")
            w = O.width2(int(o1[m, c]), int(o2[m, c]), L)
            assert abs(gw[m, j] - w) <= 1e-9 * max(1.0, w)
    for j in height_lanes:
        c = lanes.index(j)
        assert np.array_equal(gh[j], oh[c]), f"heights of lane {j} differ"
    return gts, g1, g2, gw

"""Batches: many independent jobs of different L, N and widths advanced by one
multi-job persistent launch per class (captured in a CUDA graph).  Every job's
result must be bit-identical to the same job run alone, in graph and direct
mode, and equal to the oracle on sampled lanes."""
import os

import numpy as np
import pytest

import paper_1605_02620_gb300 as R
from rsos_testlib import gpu_run, oracle_run

pytestmark = pytest.mark.gpu

JOBS = [  # (L, N, S, t_max, seed)
    (64, 1, 64, 40, 0), (128, 2, 64, 25, 1), (64, 3, 32, 30, 2), (96, 1, 64, 33, 3),
    (32, 4, 96, 20, 4), (128, 1, 64, 12, 5), (48, 2, 32, 41, 6), (64, 1, 64, 1, 7),
    (256, 1, 1, 15, 8),  # plain single surface: runs through its own handle
]


def _run_batch(jobs, graph=True, schedules=None):
    import torch
    old = os.environ.get("RSOS_BATCH_GRAPH")
    os.environ["RSOS_BATCH_GRAPH"] = "1" if graph else "0"
    try:
        params = [R.rsos_params(L=L, N=N, surfaces=S, tile=8, seed=seed, series_capacity=16)
                  for (L, N, S, t, seed) in jobs]
        b = R.rsos_batch_create(params, [t for (_, _, _, t, _) in jobs])
        try:
            for k, times in (schedules or {}).items():
                R.rsos_batch_schedule(b, k, times)
            stream = torch.cuda.Stream()
            R.rsos_batch_run(b, stream)
            done = set()
            for _ in range(200000):
                rc, ids = R.rsos_batch_poll(b)
                done |= set(ids)
                if len(done) == len(jobs):
                    break
            assert len(done) == len(jobs)
            out = []
            for k, (L, N, S, t, seed) in enumerate(jobs):
                h = R.rsos_batch_job(b, k)
                out.append(R.rsos_read_series(h, S, 16))
            return out
        finally:
            R.rsos_batch_free(b)
    finally:
        if old is None:
            del os.environ["RSOS_BATCH_GRAPH"]
        else:
            os.environ["RSOS_BATCH_GRAPH"] = old


@pytest.mark.parametrize("graph", [True, False])
def test_batch_equals_jobs_run_alone(graph):
    res = _run_batch(JOBS, graph=graph)
    for (L, N, S, t, seed), (ts, s1, s2, w2) in zip(JOBS, res):
        assert list(ts) == [t]
        _, a1, a2, _, _ = gpu_run(L, N, S, 8, seed=seed, times=[t], t_end=t)
        assert (s1 == a1).all() and (s2 == a2).all(), (L, N, S, t, seed)


def test_batch_against_oracle_and_schedules():
    sched = {0: [1, 5, 17, 40], 2: [3, 30], 6: [0, 2, 41]}
    res = _run_batch(JOBS, graph=True, schedules=sched)
    for k in (0, 2, 6):
        L, N, S, t, seed = JOBS[k]
        ts, s1, s2, _ = res[k]
        assert list(ts) == sched[k]
        ots, o1, o2, _ = oracle_run(L, N, [0, S - 1], 8, seed=seed, times=sched[k], t_end=t)
        for m in range(len(ts)):
            assert int(s1[m, 0]) == o1[m][0] and int(s1[m, S - 1]) == o1[m][1]
            assert int(s2[m, 0]) == o2[m][0] and int(s2[m, S - 1]) == o2[m][1]


def test_batch_budget_is_enforced():
    params = [R.rsos_params(L=4096, N=1, surfaces=64) for _ in range(4)]
    need = sum(R.rsos_required_bytes(p) for p in params)
    with pytest.raises(R.RsosError) as e:
        R.rsos_batch_create(params, [10] * 4, hbm_budget=need // 2)
    assert e.value.status == R.RSOS_ENOMEM

"""rsos_advance and the continuous-batching server: jobs advanced together
(and admitted while others run) give results bit-identical to each job run
alone."""
import pytest

import paper_1605_02620_gb300 as R
from paper_1605_02620_gb300.serve import Request, Server
from rsos_testlib import gpu_run

pytestmark = pytest.mark.gpu


def test_advance_equals_solo_runs_with_schedules():
    specs = [(64, 1, 64, 9, [3, 9, 20]), (128, 2, 64, 11, [20]), (96, 3, 32, 12, [1, 2, 20]),
             (64, 1, 1, 13, [20]), (256, 1, 64, 14, [5, 20])]
    hs = []
    for (L, N, S, seed, times) in specs:
        h = R.rsos_init(R.rsos_params(L=L, N=N, surfaces=S, tile=8, seed=seed, series_capacity=8))
        R.rsos_schedule(h, times)
        hs.append(h)
    try:
        R.rsos_advance(hs, [7] * len(hs))
        R.rsos_advance(hs, [20] * len(hs))
        for h, (L, N, S, seed, times) in zip(hs, specs):
            ts, s1, s2, _ = R.rsos_read_series(h, S, 8)
            gts, g1, g2, _, _ = gpu_run(L, N, S, 8, seed=seed, times=times, t_end=20)
            assert list(ts) == list(gts)
            assert (s1 == g1).all() and (s2 == g2).all()
    finally:
        for h in hs:
            R.rsos_free(h)


def test_served_results_equal_solo_runs():
    reqs = [Request(L=L, N=N, t_max=t, seed=k, surfaces=64, arrival=0.002 * k, rid=k)
            for k, (L, N, t) in enumerate([(128, 1, 30), (64, 2, 50), (256, 1, 20), (64, 4, 40), (128, 3, 25),
                                           (96, 1, 60), (64, 1, 10), (128, 2, 35), (256, 2, 15), (64, 3, 45)])]
    budget = 3 * R.rsos_required_bytes(R.rsos_params(L=256, N=2, surfaces=64, series_capacity=2))
    # epochs of a few sweeps per job, so that a job stays resident over several
    # epochs and later arrivals join it
    rep = Server(hbm_budget=budget, epoch_s=1e-5, rate_guess=1e11).run(reqs)
    assert len(rep.results) == len(reqs)
    by_id = {r.rid: r for r in rep.results}
    for q in reqs:
        _, g1, g2, _, _ = gpu_run(q.L, q.N, q.surfaces, 8, seed=q.seed, times=[q.t_max], t_end=q.t_max)
        r = by_id[q.rid]
        assert (r.sum_h == g1[0]).all() and (r.sum_h2 == g2[0]).all(), q
        assert r.finished >= r.admitted >= q.arrival - 1e-9
    s = rep.summary()
    assert s["jobs"] == len(reqs) and s["latency_p99_s"] >= s["latency_p50_s"]
    # continuous batching: jobs were resident together, and some request was
    # admitted while another job was already resident (it joined the running
    # work instead of waiting for it to drain)
    assert rep.max_active > 1
    res = rep.results
    assert any(a.admitted < b.admitted < a.finished for a in res for b in res if a is not b)

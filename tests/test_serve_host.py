"""Host logic of the serving loop with a fake device library: first-come
first-served admission under the memory budget, retirement, latency and
throughput accounting, and faults that stay with their jobs — rejected,
cancelled (queued or resident) and failed requests (an injected rsos_init or
rsos_advance error) while the other jobs finish exactly (no GPU)."""
import pytest

import paper_1605_02620_gb300.serve as S


class FakeLib:
    def __init__(self):
        self.t = {}
        self.live = 0
        self.max_live = 0
        self.n = 0
        self.fail_init_seeds = set()   # rsos_init raises for these seeds
        self.fail_advance_calls = set()  # the k-th rsos_advance call raises
        self.advance_calls = 0

    def required_bytes(self, p):
        return p.L * p.L

    def init(self, p, stream=None):
        if p.seed in self.fail_init_seeds:
            raise S.RsosError(-2, "rsos_init")  # RSOS_ENOMEM
        self.n += 1
        h = ("h", self.n)
        self.t[h] = 0
        self.live += 1
        self.max_live = max(self.max_live, self.live)
        return h

    def schedule(self, h, times):
        pass

    def time(self, h):
        return self.t[h]

    def advance(self, hs, targets, stream=None):
        self.advance_calls += 1
        if self.advance_calls in self.fail_advance_calls:
            raise S.RsosError(-5, "rsos_advance")  # RSOS_ETIMEOUT
        for h, tt in zip(hs, targets):
            assert tt >= self.t[h]
            self.t[h] = tt

    def read_series(self, h, surfaces, cap, stream=None):
        import numpy as np
        v = np.full((1, surfaces), self.t[h], dtype=np.int64)
        return np.array([self.t[h]]), v, v * v, v.astype(float)

    def free(self, h):
        del self.t[h]
        self.live -= 1


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    monkeypatch.setattr(S, "rsos_required_bytes", f.required_bytes)
    monkeypatch.setattr(S, "rsos_init", f.init)
    monkeypatch.setattr(S, "rsos_schedule", f.schedule)
    monkeypatch.setattr(S, "rsos_time", f.time)
    monkeypatch.setattr(S, "rsos_advance", f.advance)
    monkeypatch.setattr(S, "rsos_read_series", f.read_series)
    monkeypatch.setattr(S, "rsos_free", f.free)
    return f


def test_budget_limits_resident_jobs_and_all_finish(fake):
    reqs = [S.Request(L=64, N=1, t_max=10 + k, seed=k, surfaces=32, arrival=0.0, rid=k) for k in range(7)]
    srv = S.Server(hbm_budget=3 * 64 * 64, epoch_s=1.0, rate_guess=64 * 64 * 32 * 4)
    rep = srv.run(reqs, clock=iter(range(100000)).__next__, sleep=lambda s: None)
    assert sorted(r.rid for r in rep.results) == list(range(7))
    assert fake.max_live == 3 and fake.live == 0
    for r in rep.results:
        assert int(r.sum_h[0]) == 10 + r.rid  # ran exactly to t_max


def _run(reqs, budget, rate=64 * 64 * 32 * 4):
    srv = S.Server(hbm_budget=budget, epoch_s=1.0, rate_guess=rate)
    return srv.run(reqs, clock=iter(range(100000)).__next__, sleep=lambda s: None)


def _by_id(rep):
    return {r.rid: r for r in rep.results}


def test_request_larger_than_budget_is_rejected_others_finish(fake):
    reqs = [S.Request(L=64, N=1, t_max=5, seed=0, surfaces=32, rid=0),
            S.Request(L=128, N=1, t_max=5, seed=1, surfaces=32, rid=1),  # 4x the budget
            S.Request(L=64, N=1, t_max=6, seed=2, surfaces=32, rid=2)]
    rep = _run(reqs, budget=64 * 64)
    by = _by_id(rep)
    assert by[1].status == "rejected" and by[1].sum_h is None and "budget" in by[1].error
    assert by[0].status == by[2].status == "done"
    assert int(by[0].sum_h[0]) == 5 and int(by[2].sum_h[0]) == 6
    assert rep.summary()["rejected"] == 1 and rep.summary()["jobs"] == 2
    assert fake.live == 0


def test_cancelled_queued_and_resident_jobs_release_memory(fake):
    # budget for one job at a time: job 0 runs long, job 1 waits in the queue
    # and is cancelled there, job 2 is cancelled while resident
    reqs = [S.Request(L=64, N=1, t_max=400, seed=0, surfaces=32, rid=0, cancel_at=None),
            S.Request(L=64, N=1, t_max=5, seed=1, surfaces=32, rid=1, cancel_at=3.0),
            S.Request(L=64, N=1, t_max=10 ** 6, seed=2, surfaces=32, rid=2, arrival=1.0, cancel_at=200.0)]
    rep = _run(reqs, budget=64 * 64, rate=64 * 64 * 32 * 10)
    by = _by_id(rep)
    assert by[0].status == "done" and int(by[0].sum_h[0]) == 400
    assert by[1].status == "cancelled" and by[1].admitted is None
    assert by[2].status == "cancelled" and by[2].admitted is not None
    assert fake.live == 0 and fake.max_live == 1
    assert rep.summary()["cancelled"] == 2


def test_failed_init_fails_only_its_request(fake):
    fake.fail_init_seeds = {1}
    reqs = [S.Request(L=64, N=1, t_max=7 + k, seed=k, surfaces=32, rid=k) for k in range(4)]
    rep = _run(reqs, budget=2 * 64 * 64)
    by = _by_id(rep)
    assert by[1].status == "failed" and "rsos_init" in by[1].error
    for k in (0, 2, 3):
        assert by[k].status == "done" and int(by[k].sum_h[0]) == 7 + k
    assert fake.live == 0


def test_failed_epoch_releases_its_jobs_and_the_queue_carries_on(fake):
    fake.fail_advance_calls = {2}
    reqs = [S.Request(L=64, N=1, t_max=50, seed=k, surfaces=32, rid=k) for k in range(2)] + \
           [S.Request(L=64, N=1, t_max=9, seed=9, surfaces=32, rid=9, arrival=5.0)]
    rep = _run(reqs, budget=2 * 64 * 64, rate=64 * 64 * 32 * 8)
    by = _by_id(rep)
    assert by[0].status == by[1].status == "failed" and "rsos_advance" in by[0].error
    assert by[9].status == "done" and int(by[9].sum_h[0]) == 9
    assert fake.live == 0 and rep.summary()["failed"] == 2


def test_fcfs_admission_order(fake):
    reqs = [S.Request(L=64, N=1, t_max=4, seed=k, surfaces=32, arrival=float(k), rid=k) for k in range(5)]
    srv = S.Server(hbm_budget=64 * 64, epoch_s=1.0, rate_guess=64 * 64 * 32)
    rep = srv.run(reqs, clock=iter(range(100000)).__next__, sleep=lambda s: None)
    admitted = [r.admitted for r in sorted(rep.results, key=lambda r: r.rid)]
    assert admitted == sorted(admitted)

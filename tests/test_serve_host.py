"""Host logic of the serving loop with a fake device library: first-come
first-served admission under the memory budget, retirement, latency and
throughput accounting (no GPU)."""
import pytest

import paper_1605_02620_gb300.serve as S


class FakeLib:
    def __init__(self):
        self.t = {}
        self.live = 0
        self.max_live = 0
        self.n = 0

    def required_bytes(self, p):
        return p.L * p.L

    def init(self, p, stream=None):
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
        for h, tt in zip(hs, targets):
            assert tt >= self.t[h]
            self.t[h] = tt

    def read_series(self, h, surfaces, cap, stream=None):
        import numpy as np
        v = np.full((1, surfaces), self.t[h], dtype=np.int64)
        return np.array([self.t[h]]), v, v * v, v.astype(float)

    def free(self, h):
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


def test_request_larger_than_budget_is_rejected(fake):
    with pytest.raises(S.RsosError):
        S.Server(hbm_budget=100).run([S.Request(L=64, N=1, t_max=5, seed=0)], clock=iter(range(1000)).__next__,
                                     sleep=lambda s: None)


def test_fcfs_admission_order(fake):
    reqs = [S.Request(L=64, N=1, t_max=4, seed=k, surfaces=32, arrival=float(k), rid=k) for k in range(5)]
    srv = S.Server(hbm_budget=64 * 64, epoch_s=1.0, rate_guess=64 * 64 * 32)
    rep = srv.run(reqs, clock=iter(range(100000)).__next__, sleep=lambda s: None)
    admitted = [r.admitted for r in sorted(rep.results, key=lambda r: r.rid)]
    assert admitted == sorted(admitted)

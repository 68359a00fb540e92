"""Continuous-batching request loop for RSOS growth jobs.

Requests (L, N, t_max, seed, surfaces, arrival time) arrive over time.  The
server keeps every admitted job's surfaces resident on the device between
steps and, in short epochs, advances all resident jobs together with
``rsos_advance`` (one multi-job persistent launch per class, so their work
overlaps on the GPU).  Between epochs it retires jobs that reached t_max
(their exact W^2 is read back and their device memory released) and admits
queued requests first-come first-served while their device memory fits the
budget.  Each job's result is bit-identical to running it alone.

Faults stay with the jobs they concern: a request larger than the whole
budget is rejected, a request whose job cannot be created (rsos_init raises)
fails alone, a request may be cancelled at a given time (queued: dropped;
resident: its memory is released at the next epoch boundary), and if an
epoch's rsos_advance raises, the jobs resident in that epoch are released and
reported failed while the queue carries on.  Every request ends with a
status: done, rejected, cancelled or failed.

Everything that computes runs in the library's kernels; this module only
decides which jobs advance how far in each epoch.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import (RsosError, rsos_advance, rsos_free, rsos_init, rsos_params, rsos_read_series, rsos_required_bytes,
               rsos_schedule, rsos_time)


@dataclass
class Request:
    L: int
    N: int
    t_max: int
    seed: int
    surfaces: int = 64
    arrival: float = 0.0
    rid: int = 0
    cancel_at: float | None = None  # cancelled by the client at this time (None: never)


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float | None  # None: never resident
    finished: float
    sum_h: np.ndarray | None  # None unless status == "done"
    sum_h2: np.ndarray | None
    w2: np.ndarray | None
    status: str = "done"  # done, rejected, cancelled, failed
    error: str = ""

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


@dataclass
class _Active:
    req: Request
    handle: object
    nbytes: int
    admitted: float


@dataclass
class Report:
    results: list = field(default_factory=list)
    wall_s: float = 0.0
    gpu_busy_s: float = 0.0
    attempts: float = 0.0
    epochs: int = 0
    max_active: int = 0
    offered_attempts_per_s: float = 0.0

    def summary(self) -> dict:
        done = [r for r in self.results if r.status == "done"]
        lat = np.array([r.latency for r in done]) if done else np.zeros(1)
        return {
            "jobs": len(done),
            "rejected": sum(r.status == "rejected" for r in self.results),
            "cancelled": sum(r.status == "cancelled" for r in self.results),
            "failed": sum(r.status == "failed" for r in self.results),
            "wall_s": self.wall_s,
            "attempts_per_s": self.attempts / self.wall_s if self.wall_s > 0 else 0.0,
            "attempts_per_busy_s": self.attempts / self.gpu_busy_s if self.gpu_busy_s > 0 else 0.0,
            "offered_attempts_per_s": self.offered_attempts_per_s,
            "latency_p50_s": float(np.percentile(lat, 50)),
            "latency_p99_s": float(np.percentile(lat, 99)),
            "epochs": self.epochs,
            "max_resident_jobs": self.max_active,
        }


class Server:
    """hbm_budget: device bytes the resident jobs may hold.  epoch_s: target
    GPU time of one epoch (short epochs admit new work sooner)."""

    def __init__(self, hbm_budget: int, epoch_s: float = 0.02, stream=None, rate_guess: float = 4e12,
                 tune: bool = False):
        self.hbm_budget = int(hbm_budget)
        self.epoch_s = float(epoch_s)
        self.stream = stream
        self.rate = float(rate_guess)  # attempts/s estimate, refined every epoch
        self.tune = bool(tune)  # execution geometry per job shape from rsos_autotune (cached)

    def _params(self, r: Request) -> rsos_params:
        p = rsos_params(L=r.L, N=r.N, surfaces=r.surfaces, tile=8, seed=r.seed, series_capacity=2)
        if self.tune:
            from . import rsos_autotune
            tuned, _ = rsos_autotune(p, sweeps=10, stream=self.stream)
            p.words_per_thread, p.tiles_per_lane, p.phase_lag = (tuned.words_per_thread, tuned.tiles_per_lane,
                                                                 tuned.phase_lag)
        return p

    def run(self, requests, clock=time.perf_counter, sleep=time.sleep) -> Report:
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        rep = Report()
        span = max((r.arrival for r in reqs), default=0.0)
        work = sum(float(r.L) * r.L * r.surfaces * r.t_max for r in reqs)
        rep.offered_attempts_per_s = work / span if span > 0 else float("inf")
        queue, active = [], []
        used = 0
        nxt = 0
        t_start = clock()

        def end(req, admitted, status, error=""):
            rep.results.append(Result(req.rid, req.arrival, admitted, clock() - t_start, None, None, None,
                                      status, error))

        def release(a):
            nonlocal used
            try:
                rsos_free(a.handle)
            finally:
                used -= a.nbytes

        while nxt < len(reqs) or queue or active:
            now = clock() - t_start
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                queue.append(reqs[nxt])
                nxt += 1
            # cancellations: queued requests leave the queue, resident jobs
            # release their memory at this epoch boundary
            for r in [r for r in queue if r.cancel_at is not None and r.cancel_at <= now]:
                queue.remove(r)
                end(r, None, "cancelled")
            keep = []
            for a in active:
                if a.req.cancel_at is not None and a.req.cancel_at <= now:
                    release(a)
                    end(a.req, a.admitted, "cancelled")
                else:
                    keep.append(a)
            active = keep
            # admit first-come first-served while memory allows
            while queue:
                r = queue[0]
                try:
                    p = self._params(r)
                    nbytes = rsos_required_bytes(p)
                except RsosError as e:
                    queue.pop(0)
                    end(r, None, "rejected", str(e))
                    continue
                if nbytes > self.hbm_budget:
                    queue.pop(0)
                    end(r, None, "rejected", f"needs {nbytes} bytes, more than the budget {self.hbm_budget}")
                    continue
                if used + nbytes > self.hbm_budget:
                    break
                queue.pop(0)
                try:
                    h = rsos_init(p, stream=self.stream)
                except RsosError as e:
                    end(r, None, "failed", str(e))
                    continue
                try:
                    rsos_schedule(h, [r.t_max])
                except RsosError as e:
                    rsos_free(h)
                    end(r, now, "failed", str(e))
                    continue
                active.append(_Active(r, h, nbytes, now))
                used += nbytes
            rep.max_active = max(rep.max_active, len(active))
            if not active:
                if nxt < len(reqs):
                    sleep(max(0.0, reqs[nxt].arrival - (clock() - t_start)))
                continue
            # one epoch: share ~epoch_s of GPU time between the resident jobs
            per_job = self.rate * self.epoch_s / len(active)
            targets, planned = [], 0.0
            for a in active:
                t = rsos_time(a.handle)
                unit = float(a.req.L) * a.req.L * a.req.surfaces
                step = max(1, int(per_job / unit))
                tt = min(a.req.t_max, t + step)
                targets.append(tt)
                planned += unit * (tt - t)
            e0 = clock()
            try:
                rsos_advance([a.handle for a in active], targets, self.stream)
            except RsosError as e:
                # the epoch's jobs are in an unknown state: release them all
                for a in active:
                    try:
                        release(a)
                    except RsosError:
                        pass
                    end(a.req, a.admitted, "failed", str(e))
                active = []
                continue
            dt = clock() - e0
            rep.gpu_busy_s += dt
            rep.attempts += planned
            rep.epochs += 1
            if dt > 0 and planned > 0:
                self.rate = 0.7 * self.rate + 0.3 * (planned / dt)
            # retire finished jobs
            keep = []
            for a, tt in zip(active, targets):
                if tt >= a.req.t_max:
                    ts, s1, s2, w2 = rsos_read_series(a.handle, a.req.surfaces, 2, self.stream)
                    release(a)
                    rep.results.append(Result(a.req.rid, a.req.arrival, a.admitted, clock() - t_start,
                                              s1[-1].copy(), s2[-1].copy(), w2[-1].copy()))
                else:
                    keep.append(a)
            active = keep
        rep.wall_s = clock() - t_start
        return rep

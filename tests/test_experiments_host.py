"""Experiment drivers (growth, finite-size scaling, decomposition check) with
a fake library whose widths follow exact power laws: the drivers must pass
the job parameters through, measure at the paper's times (Eq. 10) or in the
steady state, and recover the exponents put in (no GPU)."""
import math

import numpy as np
import pytest

import paper_1605_02620_gb300.experiments as E
from paper_1605_02620_gb300.inputs import paper_schedule

BETA, ALPHA = 0.24, 0.39


class FakeLib:
    """The batch calls the drivers make, on widths that follow exact power
    laws with 1% noise per job and surface."""

    def __init__(self):
        self.jobs = []
        self.batches = []

    def batch_create(self, params, t_max, hbm_budget=0):
        jobs = [{"L": p.L, "N": p.N, "S": p.surfaces, "tile": (p.tile_x, p.tile_y), "tiling": p.tiling,
                 "seed": p.seed, "times": [], "t": 0, "t_max": int(t)} for p, t in zip(params, t_max)]
        self.jobs.extend(jobs)
        self.batches.append(jobs)
        return jobs

    def batch_schedule(self, b, k, times):
        b[k]["times"] = [int(t) for t in times]

    def batch_run(self, b, stream=None):
        for j in b:
            j["t"] = j["t_max"]

    def batch_poll(self, b, cap=4096):
        return 0, list(range(len(b)))

    def batch_job(self, b, k):
        return b[k]

    def batch_free(self, b):
        pass

    def read_series(self, h, S, cap, stream=None):
        ts = np.array([t for t in h["times"] if t <= h["t"]], dtype=np.int64)
        rng = np.random.Generator(np.random.PCG64(h["seed"]))
        noise = 1.0 + 0.01 * rng.standard_normal((len(ts), S))
        t_sat = h["L"] ** (ALPHA / BETA)
        w2 = np.array([[min(float(t) ** (2 * BETA), t_sat ** (2 * BETA))] * S for t in ts]) * noise
        zeros = np.zeros_like(w2, dtype=np.int64)
        return ts, zeros, zeros, w2


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    for name in ("batch_create", "batch_schedule", "batch_run", "batch_poll", "batch_job", "batch_free",
                 "read_series"):
        monkeypatch.setattr(E, "rsos_" + name, getattr(f, name))
    return f


def test_growth_measures_at_the_paper_times_and_recovers_beta(fake):
    r = E.growth(65536, 1, 5000, surfaces=32, jobs=4, seed=3, tile=(6, 10), tiling=1)
    assert len(fake.batches) == 1 and len(fake.jobs) == 4
    assert [j["seed"] for j in fake.jobs] == [3, 4, 5, 6]  # independent jobs
    job = fake.jobs[-1]
    assert job["tile"] == (6, 10) and job["tiling"] == 1 and job["S"] == 32
    assert r["t"] == [t for t in paper_schedule(5000) if t > 0]
    late = np.array(r["beta_eff"])[np.array(r["beta_eff_t"]) > 500]
    assert late.size > 0 and abs(late.mean() - BETA) < 0.01
    assert all(e >= 0 for e in r["w2_err"])
    # the fitted exponent and its jackknife error: 1% noise on W^2 per surface
    assert r["window"] == [500.0, 5000]
    assert abs(r["beta_fit"] - BETA) < 5 * r["beta_fit_err"] + 1e-4 and 0 < r["beta_fit_err"] < 0.01
    assert abs(r["beta_eq11"] - BETA) < 0.01 and r["beta_eq11_err"] >= 0


def test_growth_rejects_too_short_runs_and_single_jobs(fake):
    with pytest.raises(ValueError, match="t_max = 5"):
        E.growth(64, 1, 5, jobs=2)
    with pytest.raises(ValueError, match="two independent jobs"):
        E.growth(64, 1, 1000, jobs=1)
    assert fake.jobs == []


def test_fss_recovers_alpha_and_starts_in_the_steady_state(fake):
    Ls = [32, 64, 128, 256]
    r = E.fss(Ls, N=2, surfaces=16, jobs=3, t_factor=20.0)
    assert [row["L"] for row in r["rows"]] == Ls
    assert [len(b) for b in fake.batches] == [3] * 4
    for batch, L in zip(fake.batches, Ls):
        for job in batch:
            assert job["N"] == 2 and job["times"][0] >= 20.0 * L ** 1.61  # past L^z
            assert len(job["times"]) == 40
    assert r["alpha_eff"] == pytest.approx([ALPHA] * 3, abs=0.01)
    assert r["alpha_fit"] == pytest.approx(ALPHA, abs=0.01)
    assert 0 < r["alpha_fit_err"] < 0.01 and len(r["alpha_eff_err"]) == 3
    assert all(math.isfinite(row["S"]) and math.isfinite(row["Q"]) for row in r["rows"])


def test_decomposition_check_runs_every_tiling(fake):
    tilings = [E.parse_tiling(s) for s in ("8x8", "16x16", "6x10+1")]
    assert tilings == [(8, 0), (16, 0), ((6, 10), 1)]
    r = E.dd_consistency([64, 128], tilings, surfaces=8, jobs=2)
    assert len(r["tilings"]) == 3
    seen = [(j["tile"], j["tiling"]) for j in fake.jobs]
    assert seen == [((8, 8), 0)] * 4 + [((16, 16), 0)] * 4 + [((6, 10), 1)] * 4
    for res in r["tilings"]:
        assert res["alpha_fit"] == pytest.approx(ALPHA, abs=0.01)


def test_cli_prints_one_json_line(fake, capsys):
    E.main(["fss", "--Ls", "32", "64", "--surfaces", "8", "--jobs", "2", "--tiling", "6x10+1"])
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    import json
    d = json.loads(out[0])
    assert d["tiling"] == 1 and len(d["rows"]) == 2


def test_parse_tiling_rejects_garbage():
    with pytest.raises(ValueError):
        E.parse_tiling("6x10x3")

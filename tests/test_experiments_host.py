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
    def __init__(self):
        self.jobs = []

    def init(self, p, stream=None):
        job = {"L": p.L, "N": p.N, "S": p.surfaces, "tile": (p.tile_x, p.tile_y), "tiling": p.tiling,
               "seed": p.seed, "times": [], "t": 0}
        self.jobs.append(job)
        return job

    def schedule(self, h, times):
        h["times"] = [int(t) for t in times]

    def sweep(self, h, n, stream=None):
        h["t"] += n

    def read_series(self, h, S, cap, stream=None):
        ts = np.array([t for t in h["times"] if t <= h["t"]], dtype=np.int64)
        rng = np.random.Generator(np.random.PCG64(h["seed"]))
        noise = 1.0 + 0.01 * rng.standard_normal((len(ts), S))
        t_sat = h["L"] ** (ALPHA / BETA)
        w2 = np.array([[min(float(t) ** (2 * BETA), t_sat ** (2 * BETA))] * S for t in ts]) * noise
        zeros = np.zeros_like(w2, dtype=np.int64)
        return ts, zeros, zeros, w2

    def free(self, h):
        pass


@pytest.fixture
def fake(monkeypatch):
    f = FakeLib()
    monkeypatch.setattr(E, "rsos_init", f.init)
    monkeypatch.setattr(E, "rsos_schedule", f.schedule)
    monkeypatch.setattr(E, "rsos_sweep", f.sweep)
    monkeypatch.setattr(E, "rsos_read_series", f.read_series)
    monkeypatch.setattr(E, "rsos_free", f.free)
    return f


def test_growth_measures_at_the_paper_times_and_recovers_beta(fake):
    r = E.growth(65536, 1, 5000, surfaces=32, seed=3, tile=(6, 10), tiling=1)
    job = fake.jobs[-1]
    assert job["tile"] == (6, 10) and job["tiling"] == 1 and job["S"] == 32
    assert r["t"] == [t for t in paper_schedule(5000) if t > 0]
    late = np.array(r["beta_eff"])[np.array(r["beta_eff_t"]) > 500]
    assert late.size > 0 and abs(late.mean() - BETA) < 0.01
    assert all(e >= 0 for e in r["w2_err"])


def test_fss_recovers_alpha_and_starts_in_the_steady_state(fake):
    Ls = [32, 64, 128, 256]
    r = E.fss(Ls, N=2, surfaces=16, t_factor=20.0)
    assert [row["L"] for row in r["rows"]] == Ls
    for job, L in zip(fake.jobs, Ls):
        assert job["N"] == 2 and job["times"][0] >= 20.0 * L ** 1.61  # past L^z
        assert len(job["times"]) == 40
    assert r["alpha_eff"] == pytest.approx([ALPHA] * 3, abs=0.01)
    assert r["alpha_fit"] == pytest.approx(ALPHA, abs=0.01)
    assert all(math.isfinite(row["S"]) and math.isfinite(row["Q"]) for row in r["rows"])


def test_decomposition_check_runs_every_tiling(fake):
    tilings = [E.parse_tiling(s) for s in ("8x8", "16x16", "6x10+1")]
    assert tilings == [(8, 0), (16, 0), ((6, 10), 1)]
    r = E.dd_consistency([64, 128], tilings, surfaces=8)
    assert len(r["tilings"]) == 3
    seen = [(j["tile"], j["tiling"]) for j in fake.jobs]
    assert seen == [((8, 8), 0)] * 2 + [((16, 16), 0)] * 2 + [((6, 10), 1)] * 2
    for res in r["tilings"]:
        assert res["alpha_fit"] == pytest.approx(ALPHA, abs=0.01)


def test_cli_prints_one_json_line(fake, capsys):
    E.main(["fss", "--Ls", "32", "64", "--surfaces", "8", "--tiling", "6x10+1"])
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    import json
    d = json.loads(out[0])
    assert d["tiling"] == 1 and len(d["rows"]) == 2


def test_parse_tiling_rejects_garbage():
    with pytest.raises(ValueError):
        E.parse_tiling("6x10x3")

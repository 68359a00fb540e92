"""JSONL records keep exact sums of any size and every (time, surface)."""
import numpy as np

from paper_1605_02620_gb300 import records


def test_round_trip_exact(tmp_path):
    big = (1 << 100) + 12345
    times = [0, 5]
    s1 = np.array([[0, 0], [7, -3]], dtype=object)
    s2 = np.array([[0, 0], [big, 9]], dtype=object)
    w2 = np.array([[0.0, 0.0], [0.25, 1.5]])
    mom = np.array([[[0, 0, 0, 0], [0, 0, 0, 0]], [[7, big, -big, big * big], [-3, 9, -27, 81]]], dtype=object)
    path = str(tmp_path / "job.jsonl")
    assert records.write_series(path, {"L": 64, "N": 1, "seed": 3}, times, s1, s2, w2, mom, append=False) == 4
    rows = records.read_series(path)
    assert [(r["t"], r["surface"]) for r in rows] == [(0, 0), (0, 1), (5, 0), (5, 1)]
    assert rows[2]["sum_h2"] == big and rows[2]["sum_h3"] == -big and rows[2]["sum_h4"] == big * big
    assert rows[3]["w2"] == 1.5 and rows[3]["L"] == 64

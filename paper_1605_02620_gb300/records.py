"""Per-job measurement records as JSON lines: one line per (time, surface)
with the exact sums (as decimal strings, so any size survives JSON) and W^2.
Host-side formatting of what rsos_read_series / rsos_read_moments return."""
from __future__ import annotations

import json


def series_lines(job: dict, times, sum_h, sum_h2, w2, moments=None):
    """Yield one JSON line per (time, surface).  job: free-form identifying
    fields (L, N, seed, ...); moments: optional [n][S][4] exact power sums."""
    for m, t in enumerate(times):
        for j in range(len(sum_h[m])):
            rec = dict(job, t=int(t), surface=j, sum_h=str(int(sum_h[m][j])), sum_h2=str(int(sum_h2[m][j])),
                       w2=float(w2[m][j]))
            if moments is not None:
                rec["sum_h3"] = str(int(moments[m][j][2]))
                rec["sum_h4"] = str(int(moments[m][j][3]))
            yield json.dumps(rec, sort_keys=True)


def write_series(path: str, job: dict, times, sum_h, sum_h2, w2, moments=None, append: bool = True) -> int:
    """Append (or write) the records of one job to a JSONL file; returns the
    number of lines."""
    n = 0
    with open(path, "a" if append else "w") as f:
        for line in series_lines(job, times, sum_h, sum_h2, w2, moments):
            f.write(line + "\n")
            n += 1
    return n


def read_series(path: str):
    """Records of a JSONL file, sums back as Python ints."""
    out = []
    with open(path) as f:
        for line in f:
            r = json.loads(line)
            for k in ("sum_h", "sum_h2", "sum_h3", "sum_h4"):
                if k in r:
                    r[k] = int(r[k])
            out.append(r)
    return out

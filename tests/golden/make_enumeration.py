"""Writes tests/golden/enumeration.json: exact stationary growth velocity and
squared width (Eq. 2) of RSOS chains (Eq. 6) on tiny periodic lattices, for the
random-sequential and the double-tiling dynamics (section II), and for double
tiling on the (+1) tilings of section III.C.

Calls only oracle.enumerate.  Run:  python tests/golden/make_enumeration.py
(``--only dt_general`` recomputes that section and keeps the others.)
"""
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
from oracle import enumerate as en  # noqa: E402

CASES_RS = [(2, 1), (2, 2), (3, 1), (3, 2)]
CASES_DT = [(2, 1, 2, 0), (2, 2, 2, 0), (2, 1, 2, 1), (2, 3, 2, 0), (4, 1, 2, 1), (4, 1, 4, 1), (4, 1, 2, 0)]
# (+1) tilings: L = 3 with base edge 2 is one 3-site tile per axis, halved
# into 1 + 2 sites; the origin is uniform over the 3 x 3 lattice.
CASES_DT_GENERAL = [(3, 1, 2, 2, 0), (3, 1, 2, 2, 1), (3, 2, 2, 2, 1)]


def main():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "enumeration.json")
    only = sys.argv[sys.argv.index("--only") + 1] if "--only" in sys.argv else None
    if only:
        with open(path) as f:
            out = json.load(f)
    else:
        out = {"source": "oracle/enumerate.py (exact power iteration, tol 1e-14)", "rs": [], "dt": []}
    if only is None:
        for L, N in CASES_RS:
            t = time.time()
            out["rs"].append(en.rs_chain(L, N))
            print("rs", L, N, round(time.time() - t, 1), "s", flush=True)
        for L, N, T, order in CASES_DT:
            t = time.time()
            out["dt"].append(en.dt_chain(L, N, T, T, order))
            print("dt", L, N, T, order, round(time.time() - t, 1), "s", flush=True)
    if only in (None, "dt_general"):
        out["dt_general"] = []
        for L, N, Tx, Ty, order in CASES_DT_GENERAL:
            t = time.time()
            out["dt_general"].append(en.dt_chain_general(L, N, Tx, Ty, order))
            print("dt_general", L, N, Tx, Ty, order, round(time.time() - t, 1), "s", flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()

"""Pins for the oracle's constraint checker orc_max_step: the largest
|h(x) - h(n)| over all nearest-neighbour pairs of a periodic field (the
quantity Eq. 6 bounds by N).  The invariant tests rely on it, so it is pinned
here on hand-built fields whose answer is known by construction: a step
along x only, along y only, across the periodic wrap in each direction, and
fields whose largest step appears only as a negative forward difference (a
checker that forgets the absolute value, a direction or the wrap fails one
of them).  Random fields are checked against a brute force over the four
neighbour shifts."""
import numpy as np
import pytest

import oracle as O


def hand_built_cases():
    """(name, field[L][L], expected max step) built so that the answer is
    known by construction."""
    cases = [("flat", np.zeros((6, 6)), 0), ("flat, far from zero", np.full((5, 5), 123456789), 0)]
    for L in (4, 7):
        for N in (1, 2, 4):
            f = np.zeros((L, L))
            f[2, 1] = N + 1  # a deposit of N + 1 on a flat field
            cases.append((f"raised site L={L} N={N}", f, N + 1))
    L = 8
    f = np.zeros((L, L))
    f[:, 3] = 5  # raised column: only horizontal pairs differ
    cases.append(("step along x only", f, 5))
    g = np.zeros((L, L))
    g[2, :] = 7  # raised row: only vertical pairs differ
    cases.append(("step along y only", g, 7))
    L = 9
    x = np.arange(L)
    # ramps: every interior step is 1, the wrap from the last column (row) to the first is L - 1
    cases.append(("wrap along x", np.tile(x, (L, 1)), L - 1))
    cases.append(("wrap along y", np.tile(x[:, None], (1, L)), L - 1))
    # h = -x: forward differences h(x) - h(x+1) are +1 inside and -(L-1) at the wrap
    cases.append(("negative wrap along x", -np.tile(x, (L, 1)), L - 1))
    cases.append(("negative wrap along y", -np.tile(x[:, None], (1, L)), L - 1))
    # a staircase whose one large step goes down in the forward direction, away from the wrap
    row = np.array([0] + list(range(L - 1, 0, -1)))
    cases.append(("negative step along x", np.tile(row, (L, 1)), L - 1))
    cases.append(("negative step along y", np.tile(row[:, None], (1, L)), L - 1))
    f = np.zeros((6, 6))
    f[4, 4] = -3
    cases.append(("pit", f.copy(), 3))
    f[0, 0] = 10 ** 12  # heights far from zero: no overflow in the differences
    cases.append(("tall site", f, 10 ** 12))
    return [(n, np.ascontiguousarray(np.asarray(a, dtype=np.int64)), e) for n, a, e in cases]


def one(field, max_step=O.max_step):
    return int(max_step(np.ascontiguousarray(field[None]))[0])


@pytest.mark.parametrize("name,field,expected", hand_built_cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_hand_built_field(name, field, expected):
    assert one(field) == expected, name


def test_each_field_of_a_batch_is_separate():
    L = 5
    h = np.zeros((3, L, L), dtype=np.int64)
    h[1, 2, 2] = 4
    h[2, :, 0] = -6
    assert list(O.max_step(h)) == [0, 4, 6]


def test_random_fields_against_brute_force():
    rng = np.random.Generator(np.random.PCG64(605))
    for L in (2, 3, 5, 16):
        h = rng.integers(-50, 50, size=(4, L, L)).astype(np.int64)
        want = [max(int(np.abs(f - np.roll(f, s, axis=a)).max()) for a in (0, 1) for s in (1, -1)) for f in h]
        assert list(O.max_step(h)) == want

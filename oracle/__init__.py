"""CPU oracle for the RSOS double-tiling sweep (test infrastructure only).

This package is the reference the CUDA path is checked against.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it.  It shares no code with ``paper_1605_02620_gb300`` and imports
nothing from it.

* ``rsos_oracle.c``  -- Philox-4x32-10, the double-tiling (DT) sweep and the
  random-sequential (RS) step of Eq. 6 on int64 heights, exact sums (Eq. 2)
  and power sums up to the fourth (height-distribution moments, §III.C).
* ``enumerate.py``   -- exact Markov-chain enumeration on tiny lattices.

The C file is compiled with gcc on first use (``build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsos_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle C file into ``oracle/_build/liboracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32p = ctypes.POINTER(ctypes.c_uint32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.orc_philox4x32_10.restype = None
            lib.orc_philox_constants.argtypes = [u32p]
            lib.orc_philox_constants.restype = None
            lib.orc_philox_bulk.argtypes = [u32p, u32p, ctypes.c_uint64, u32p]
            lib.orc_philox_bulk.restype = None
            lib.orc_control.argtypes = [ctypes.c_void_p, ctypes.c_uint64, i32p, i32p, i32p]
            lib.orc_control.restype = None
            lib.orc_axis_half.argtypes = [ctypes.c_int32] * 4 + [i32p, i32p]
            lib.orc_axis_half.restype = None
            lib.orc_sweeps.argtypes = [ctypes.c_void_p, i64p, u32p, ctypes.c_int32, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, i64p]
            lib.orc_sweeps.restype = ctypes.c_int
            lib.orc_sums.argtypes = [i64p, ctypes.c_int32, ctypes.c_int32, i64p, i64p, u64p]
            lib.orc_sums.restype = None
            lib.orc_power_sums.argtypes = [i64p, ctypes.c_int32, ctypes.c_int32, i64p]
            lib.orc_power_sums.restype = None
            lib.orc_max_step.argtypes = [i64p, ctypes.c_int32, ctypes.c_int32, i64p]
            lib.orc_max_step.restype = None
            _lib = lib
    return _lib


class _Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("N", ctypes.c_int32), ("Tx", ctypes.c_int32),
                ("Ty", ctypes.c_int32), ("phase_order", ctypes.c_int32), ("tiling", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


@dataclass(frozen=True)
class Params:
    """Model parameters: lattice edge L, step bound N (Eq. 6), DT tile Tx x Ty
    (section II; 8 x 8 in the paper's runs), phase order (0: random per sweep,
    1: fixed 0,1,2,3), the Philox key, and the tiling: 0 for regular tiles
    (Tx, Ty even, dividing L), 1 for the (+1) tilings of section III.C (tiles
    Tx or Tx + 1 wide, Ty or Ty + 1 high)."""
    L: int
    N: int
    Tx: int = 8
    Ty: int = 8
    phase_order: int = 0
    seed: int = 0
    tiling: int = 0

    def c(self) -> _Params:
        return _Params(self.L, self.N, self.Tx, self.Ty, self.phase_order, self.tiling,
                       self.seed & 0xFFFFFFFFFFFFFFFF)


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def philox4x32_10(ctr, key) -> np.ndarray:
    """One Philox-4x32-10 block: 4 counter words, 2 key words -> 4 words."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), _ptr(out, ctypes.c_uint32))
    return out


def philox_constants() -> tuple:
    """(M0, M1, W0, W1) as compiled into the oracle."""
    lib = _load()
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox_constants(_ptr(out, ctypes.c_uint32))
    return tuple(int(v) for v in out)


def philox_bulk(ctr0, key, n: int) -> np.ndarray:
    """n consecutive Philox blocks (counter words 0-1 as a 64-bit count from
    ctr0), as a [n, 4] uint32 array."""
    lib = _load()
    c = np.ascontiguousarray(ctr0, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros((n, 4), dtype=np.uint32)
    lib.orc_philox_bulk(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32), n, _ptr(out, ctypes.c_uint32))
    return out


def control(p: Params, t: int):
    """Tiling origin (ox, oy) and phase permutation of sweep t."""
    lib = _load()
    ox, oy = ctypes.c_int32(), ctypes.c_int32()
    perm = np.zeros(4, dtype=np.int32)
    pc = p.c()
    lib.orc_control(ctypes.byref(pc), t, ctypes.byref(ox), ctypes.byref(oy), _ptr(perm, ctypes.c_int32))
    return ox.value, oy.value, tuple(int(v) for v in perm)


def axis_half(L: int, T: int, c: int, half: int):
    """(start, width) in pattern coordinates of half `half` of tile c along an
    axis of a (+1) tiling with base edge T (section III.C)."""
    lib = _load()
    a, w = ctypes.c_int32(), ctypes.c_int32()
    lib.orc_axis_half(L, T, c, half, ctypes.byref(a), ctypes.byref(w))
    return a.value, w.value


def flat(L: int, n_lanes: int) -> np.ndarray:
    """Flat initial condition (section II): all heights zero."""
    return np.zeros((n_lanes, L, L), dtype=np.int64)


def sweeps(p: Params, h: np.ndarray, lanes, t0: int, n: int, rs: bool = False,
           threads: int | None = None) -> np.ndarray:
    """Advance the fields h[m] (lane lanes[m]) in place by n sweeps from sweep
    index t0 (DT), or by n Monte-Carlo steps (RS).  Returns accepted deposits."""
    lib = _load()
    assert h.dtype == np.int64 and h.flags.c_contiguous and h.shape[1:] == (p.L, p.L)
    ln = np.ascontiguousarray(lanes, dtype=np.uint32)
    assert ln.shape == (h.shape[0],)
    acc = np.zeros(h.shape[0], dtype=np.int64)
    if threads is None:
        # DT sweeps run the tile rows of a sub-tile set in parallel; RS steps
        # one lane per thread
        threads = os.cpu_count() or 1
        if rs:
            threads = max(1, min(threads, h.shape[0]))
    pc = p.c()
    rc = lib.orc_sweeps(ctypes.byref(pc), _ptr(h, ctypes.c_int64), _ptr(ln, ctypes.c_uint32),
                        h.shape[0], t0, n, 1 if rs else 0, threads, _ptr(acc, ctypes.c_int64))
    if rc != 0:
        raise ValueError("invalid oracle parameters")
    return acc


def sums(h: np.ndarray):
    """Exact (sum h, sum h^2) per field as Python ints (Eq. 2 numerators)."""
    lib = _load()
    assert h.dtype == np.int64 and h.flags.c_contiguous
    n, L = h.shape[0], h.shape[1]
    s1 = np.zeros(n, dtype=np.int64)
    hi = np.zeros(n, dtype=np.int64)
    lo = np.zeros(n, dtype=np.uint64)
    lib.orc_sums(_ptr(h, ctypes.c_int64), L, n, _ptr(s1, ctypes.c_int64), _ptr(hi, ctypes.c_int64),
                 _ptr(lo, ctypes.c_uint64))
    return [int(v) for v in s1], [(int(a) << 64) + int(b) for a, b in zip(hi, lo)]


def power_sums(h: np.ndarray):
    """Exact [sum h, sum h^2, sum h^3, sum h^4] per field as Python ints."""
    lib = _load()
    assert h.dtype == np.int64 and h.flags.c_contiguous
    n, L = h.shape[0], h.shape[1]
    w = np.zeros((n, 8), dtype=np.int64)
    lib.orc_power_sums(_ptr(h, ctypes.c_int64), L, n, _ptr(w, ctypes.c_int64))
    return [[int(r[2 * k]) % (1 << 64) + (int(r[2 * k + 1]) << 64) for k in range(4)] for r in w]


def central_moments(ps, L: int):
    """Central moments (Phi^2, Phi^3, Phi^4) of one field's height distribution
    from its exact power sums (section III.C), as exact fractions."""
    from fractions import Fraction
    n = L * L
    m1, m2, m3, m4 = (Fraction(v, n) for v in ps)
    c2 = m2 - m1 * m1
    c3 = m3 - 3 * m1 * m2 + 2 * m1 ** 3
    c4 = m4 - 4 * m1 * m3 + 6 * m1 * m1 * m2 - 3 * m1 ** 4
    return c2, c3, c4


def width2(sum_h: int, sum_h2: int, L: int) -> float:
    """Eq. 2: W^2 = sum h^2 / L^2 - (sum h / L^2)^2, from exact integers."""
    area = L * L
    return (area * sum_h2 - sum_h * sum_h) / float(area * area)


def max_step(h: np.ndarray) -> np.ndarray:
    """Largest nearest-neighbour |h(x) - h(n)| per field."""
    lib = _load()
    out = np.zeros(h.shape[0], dtype=np.int64)
    lib.orc_max_step(_ptr(h, ctypes.c_int64), h.shape[1], h.shape[0], _ptr(out, ctypes.c_int64))
    return out


def run_series(p: Params, lanes, times, rs: bool = False, threads: int | None = None, powers: bool = False):
    """Run from the flat start and record exact sums at each time in ``times``
    (completed sweeps, ascending; 0 = the flat start).  Returns
    (times, sum_h[len(times)][lanes], sum_h2[...], final heights), and with
    ``powers`` also the power sums [len(times)][lanes][4] (power_sums)."""
    lanes = list(lanes)
    h = flat(p.L, len(lanes))
    t = 0
    out_s1, out_s2, out_p = [], [], []
    for T in times:
        if T < t:
            raise ValueError("times must be ascending")
        if T > t:
            sweeps(p, h, lanes, t, T - t, rs=rs, threads=threads)
            t = T
        s1, s2 = sums(h)
        out_s1.append(s1)
        out_s2.append(s2)
        if powers:
            out_p.append(power_sums(h))
    if powers:
        return list(times), out_s1, out_s2, h, out_p
    return list(times), out_s1, out_s2, h

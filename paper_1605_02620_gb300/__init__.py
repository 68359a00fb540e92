"""GB300-native RSOS multisurface sweep (Kelling, Odor & Gemming, arXiv:1605.02620).

Thin ctypes binding over the C ABI of ``include/rsos.h`` (librsos.so).  Every
function has the name of the C entry point and only marshals arguments: all
work runs in the library's CUDA kernels.  There is no CPU fallback; if the
shared library cannot be loaded (or built from source with nvcc) the first
call raises.

PyTorch is optional plumbing: a ``torch.cuda.Stream`` (or a raw cudaStream_t
integer) may be passed wherever a stream is accepted, and a CUDA tensor may be
passed as the caller-owned device buffer of ``rsos_init``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = [
    "RsosError", "rsos_params", "rsos_required_bytes", "rsos_init", "rsos_sweep", "rsos_width",
    "rsos_schedule", "rsos_read_series", "rsos_heights", "rsos_time", "rsos_free", "rsos_strerror",
    "rsos_selftest_timeout", "rsos_launches", "rsos_width_noalloc", "rsos_advance",
    "rsos_last_cuda_error", "rsos_batch_create", "rsos_batch_schedule", "rsos_batch_run",
    "rsos_batch_poll", "rsos_batch_job", "rsos_batch_free", "rsos_set_moments", "rsos_moments",
    "rsos_read_moments", "rsos_autotune", "rsos_snapshot", "rsos_restore", "rsos_snapshot_bytes",
    "rsos_peak_int", "rsos_checked_build", "rsos_bounds_errors", "library_path",
]

RSOS_OK = 0
RSOS_EINVAL = -1
RSOS_ENOMEM = -2
RSOS_ECUDA = -3
RSOS_EOVERFLOW = -4
RSOS_ETIMEOUT = -5
RSOS_EBUSY = -6
RSOS_ERANGE = -7

_HERE = os.path.dirname(os.path.abspath(__file__))
# RSOS_CHECKED=1 loads the bounds-checked build (built on first use).
_CHECKED = os.environ.get("RSOS_CHECKED", "0") == "1"
_LIB_PATH = os.path.join(_HERE, "_build_checked" if _CHECKED else "_build", "librsos.so")
_lock = threading.Lock()
_lib = None


class RsosError(RuntimeError):
    def __init__(self, status: int, what: str, cuda_error: int = 0):
        extra = f", cuda error {cuda_error}" if cuda_error else ""
        super().__init__(f"{what}: {rsos_strerror(status)} ({status}{extra})")
        self.status = status
        self.cuda_error = cuda_error


class rsos_params(ctypes.Structure):
    """Mirror of the C struct rsos_params (include/rsos.h).  ``tile`` is a
    square edge or a (Tx, Ty) pair; ``tiling=1`` selects the (+1) tilings of
    section III.C, whose Tx, Ty are base edges."""
    _fields_ = [("L", ctypes.c_int32), ("N", ctypes.c_int32), ("surfaces", ctypes.c_int32),
                ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32), ("phase_order", ctypes.c_int32),
                ("series_capacity", ctypes.c_int32), ("engine", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("words_per_thread", ctypes.c_int32), ("tiles_per_lane", ctypes.c_int32),
                ("phase_lag", ctypes.c_int32), ("tiling", ctypes.c_int32)]

    def __init__(self, L=64, N=1, surfaces=1, tile=8, phase_order=0, series_capacity=0, engine=0, seed=0,
                 words_per_thread=0, tiles_per_lane=0, phase_lag=0, tiling=0, tile_y=None):
        # tile: square edge, or (Tx, Ty); tile_y overrides the second edge
        tx, ty = (tile, tile) if not isinstance(tile, (tuple, list)) else tile
        if tile_y is not None:
            ty = tile_y
        super().__init__(int(L), int(N), int(surfaces), int(tx), int(ty), int(phase_order),
                         int(series_capacity), int(engine), int(seed) & 0xFFFFFFFFFFFFFFFF,
                         int(words_per_thread), int(tiles_per_lane), int(phase_lag), int(tiling))


def library_path() -> str:
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            from . import build as _build
            _build.build(checked=_CHECKED)
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        P = ctypes.POINTER
        sig = {
            "rsos_required_bytes": [P(rsos_params), P(sz)],
            "rsos_init": [P(rsos_params), vp, sz, vp, P(vp)],
            "rsos_sweep": [vp, i64, vp],
            "rsos_width": [vp, P(i64), P(i64), P(ctypes.c_double), P(i64), vp],
            "rsos_schedule": [vp, P(i64), i32],
            "rsos_read_series": [vp, P(i64), P(i64), P(i64), P(ctypes.c_double), i32, P(i32), vp],
            "rsos_heights": [vp, i32, P(i64), vp],
            "rsos_set_moments": [vp, i32],
            "rsos_snapshot_bytes": [vp, P(sz)],
            "rsos_snapshot": [vp, vp, sz, vp],
            "rsos_restore": [vp, sz, vp, sz, vp, P(vp)],
            "rsos_autotune": [P(rsos_params), i32, P(rsos_params), P(ctypes.c_double), vp],
            "rsos_moments": [vp, P(i64), P(i64), vp],
            "rsos_read_moments": [vp, P(i64), P(i64), P(ctypes.c_int8), i32, P(i32), vp],
            "rsos_time": [vp, P(i64)],
            "rsos_selftest_timeout": [vp, i64, vp],
            "rsos_launches": [vp, P(i64)],
            "rsos_width_noalloc": [P(rsos_params), vp, vp, vp, vp],
            "rsos_advance": [P(vp), P(i64), i32, vp],
            "rsos_free": [vp],
            "rsos_last_cuda_error": [vp],
            "rsos_batch_create": [P(rsos_params), P(i64), i32, sz, P(vp)],
            "rsos_batch_schedule": [vp, i32, P(i64), i32],
            "rsos_batch_run": [vp, vp],
            "rsos_batch_poll": [vp, P(i32), i32, P(i32)],
            "rsos_batch_job": [vp, i32, P(vp)],
            "rsos_batch_free": [vp],
            "rsos_peak_int": [i32, i64, P(ctypes.c_double), vp],
            "rsos_checked_build": [],
            "rsos_bounds_errors": [vp, P(ctypes.c_uint32), vp],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        lib.rsos_strerror.argtypes = [ctypes.c_int]
        lib.rsos_strerror.restype = ctypes.c_char_p
        _lib = lib
        return lib


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return ctypes.c_void_p(s)
    return ctypes.c_void_p(int(s.cuda_stream))  # torch.cuda.Stream


def _check(rc: int, what: str, allow=()):
    if rc != RSOS_OK and rc not in allow:
        raise RsosError(rc, what)
    return rc


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def rsos_strerror(status: int) -> str:
    return _load().rsos_strerror(int(status)).decode()


def rsos_required_bytes(params: rsos_params) -> int:
    out = ctypes.c_size_t()
    _check(_load().rsos_required_bytes(ctypes.byref(params), ctypes.byref(out)), "rsos_required_bytes")
    return out.value


def rsos_init(params: rsos_params, dev_buf=None, dev_bytes: int = 0, stream=None):
    """Create a job (flat start, t = 0).  ``dev_buf``: None (library allocates),
    an integer device address, or a CUDA tensor (its storage, which the caller
    keeps alive).  Returns the opaque handle."""
    ptr = None
    if dev_buf is not None:
        if isinstance(dev_buf, int):
            ptr = ctypes.c_void_p(dev_buf)
        else:
            ptr = ctypes.c_void_p(int(dev_buf.data_ptr()))
            if not dev_bytes:
                dev_bytes = int(dev_buf.numel() * dev_buf.element_size())
    h = ctypes.c_void_p()
    rc = _load().rsos_init(ctypes.byref(params), ptr, int(dev_bytes), _stream(stream), ctypes.byref(h))
    if rc != RSOS_OK:
        raise RsosError(rc, "rsos_init", _load().rsos_last_cuda_error(None) if rc == RSOS_ECUDA else 0)
    return h


def rsos_sweep(h, n_sweeps: int, stream=None) -> None:
    _check(_load().rsos_sweep(h, int(n_sweeps), _stream(stream)), "rsos_sweep")


def rsos_width(h, surfaces: int, stream=None, allow_overflow: bool = False):
    """Measure now.  Returns (sum_h, sum_h2, w2, t) with int64/float64 arrays of
    length ``surfaces``."""
    s1 = np.zeros(surfaces, dtype=np.int64)
    s2 = np.zeros(surfaces, dtype=np.int64)
    w2 = np.zeros(surfaces, dtype=np.float64)
    t = ctypes.c_int64()
    _check(_load().rsos_width(h, _p(s1, ctypes.c_int64), _p(s2, ctypes.c_int64), _p(w2, ctypes.c_double),
                              ctypes.byref(t), _stream(stream)),
           "rsos_width", allow=(RSOS_EOVERFLOW,) if allow_overflow else ())
    return s1, s2, w2, t.value


def rsos_schedule(h, times) -> None:
    a = np.ascontiguousarray(times, dtype=np.int64)
    _check(_load().rsos_schedule(h, _p(a, ctypes.c_int64), len(a)), "rsos_schedule")


def rsos_read_series(h, surfaces: int, cap: int, stream=None, allow_overflow: bool = False):
    """Returns (times[n], sum_h[n, S], sum_h2[n, S], w2[n, S])."""
    times = np.zeros(cap, dtype=np.int64)
    s1 = np.zeros((cap, surfaces), dtype=np.int64)
    s2 = np.zeros((cap, surfaces), dtype=np.int64)
    w2 = np.zeros((cap, surfaces), dtype=np.float64)
    n = ctypes.c_int32()
    _check(_load().rsos_read_series(h, _p(times, ctypes.c_int64), _p(s1, ctypes.c_int64), _p(s2, ctypes.c_int64),
                                    _p(w2, ctypes.c_double), int(cap), ctypes.byref(n), _stream(stream)),
           "rsos_read_series", allow=(RSOS_EOVERFLOW,) if allow_overflow else ())
    k = n.value
    return times[:k], s1[:k], s2[:k], w2[:k]


def _int128_rows(words: np.ndarray) -> list:
    """[..., 8] int64 words (four 128-bit (lo, hi) pairs) -> nested lists of
    four Python ints: sum h, sum h^2, sum h^3, sum h^4."""
    flat = words.reshape(-1, 8)
    out = [[int(r[2 * k]) % (1 << 64) + (int(r[2 * k + 1]) << 64) for k in range(4)] for r in flat]
    return np.array(out, dtype=object).reshape(words.shape[:-1] + (4,))


def rsos_autotune(params: rsos_params, sweeps: int = 20, stream=None):
    """Fastest execution geometry for params' job shape (cached per device and
    shape): (tuned rsos_params, microseconds per sweep)."""
    tuned = rsos_params()
    us = ctypes.c_double()
    _check(_load().rsos_autotune(ctypes.byref(params), int(sweeps), ctypes.byref(tuned), ctypes.byref(us),
                                 _stream(stream)), "rsos_autotune")
    return tuned, us.value


def rsos_snapshot_bytes(h) -> int:
    n = ctypes.c_size_t()
    _check(_load().rsos_snapshot_bytes(h, ctypes.byref(n)), "rsos_snapshot_bytes")
    return n.value


def rsos_snapshot(h, stream=None) -> bytes:
    """The job's whole state as bytes (bit-exact resume with rsos_restore)."""
    n = ctypes.c_size_t()
    _check(_load().rsos_snapshot_bytes(h, ctypes.byref(n)), "rsos_snapshot_bytes")
    buf = ctypes.create_string_buffer(n.value)
    _check(_load().rsos_snapshot(h, buf, n.value, _stream(stream)), "rsos_snapshot")
    return buf.raw


def rsos_restore(data: bytes, dev_buf: int = 0, dev_bytes: int = 0, stream=None):
    """A new handle continuing the snapshot's job."""
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check(_load().rsos_restore(buf, len(data), ctypes.c_void_p(dev_buf or None), int(dev_bytes),
                                _stream(stream), ctypes.byref(h)), "rsos_restore")
    return h


def rsos_set_moments(h, on: bool = True) -> None:
    _check(_load().rsos_set_moments(h, 1 if on else 0), "rsos_set_moments")


def rsos_moments(h, surfaces: int, stream=None):
    """Measure now with moments: (t, sums[S, 4]) with exact Python ints
    sum h, sum h^2, sum h^3, sum h^4 per surface."""
    words = np.zeros((surfaces, 8), dtype=np.int64)
    t = ctypes.c_int64()
    _check(_load().rsos_moments(h, _p(words, ctypes.c_int64), ctypes.byref(t), _stream(stream)), "rsos_moments")
    return t.value, _int128_rows(words)


def rsos_read_moments(h, surfaces: int, cap: int, stream=None):
    """The series with moments: (times[n], sums[n, S, 4] exact Python ints,
    has[n]: rows measured with moments on)."""
    times = np.zeros(cap, dtype=np.int64)
    words = np.zeros((cap, surfaces, 8), dtype=np.int64)
    has = np.zeros(cap, dtype=np.int8)
    n = ctypes.c_int32()
    _check(_load().rsos_read_moments(h, _p(times, ctypes.c_int64), _p(words, ctypes.c_int64), _p(has, ctypes.c_int8),
                                     int(cap), ctypes.byref(n), _stream(stream)), "rsos_read_moments")
    k = n.value
    return times[:k], _int128_rows(words[:k]), has[:k].astype(bool)


def rsos_heights(h, surface: int, L: int, stream=None) -> np.ndarray:
    out = np.zeros((L, L), dtype=np.int64)
    _check(_load().rsos_heights(h, int(surface), _p(out, ctypes.c_int64), _stream(stream)), "rsos_heights")
    return out


def rsos_selftest_timeout(h, budget_ns: int, stream=None) -> int:
    """Force every dependency wait of one persistent launch to expire; returns
    the status (RSOS_ETIMEOUT when the device reported the expiry)."""
    return _check(_load().rsos_selftest_timeout(h, int(budget_ns), _stream(stream)), "rsos_selftest_timeout",
                  allow=(RSOS_ETIMEOUT,))


def rsos_width_noalloc(params: rsos_params, planes: int, h00: int, sums: int, stream=None) -> None:
    """Exact sums of a multisurface lattice given by device addresses, without
    any allocation (for callers that cannot allocate; see include/rsos.h).
    ``sums`` is a device address of surfaces x 4 int64 (128-bit sum h, sum h^2)."""
    _check(_load().rsos_width_noalloc(ctypes.byref(params), ctypes.c_void_p(int(planes)), ctypes.c_void_p(int(h00)),
                                      ctypes.c_void_p(int(sums)), _stream(stream)), "rsos_width_noalloc")


def rsos_advance(handles, targets, stream=None) -> None:
    """Advance several jobs together to their target times (one multi-job
    persistent launch per class; synchronises the stream)."""
    n = len(handles)
    arr = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    tg = np.ascontiguousarray(targets, dtype=np.int64)
    rc = _load().rsos_advance(arr, _p(tg, ctypes.c_int64), n, _stream(stream))
    if rc != RSOS_OK:
        raise RsosError(rc, "rsos_advance", _load().rsos_last_cuda_error(None) if rc == RSOS_ECUDA else 0)


def rsos_peak_int(kind: int, iters: int = 4096, stream=None) -> float:
    """Measured integer throughput: kind 0 lop3 lane-ops/s, 1 mad.lo
    lane-ops/s, 2 Philox-4x32-10 blocks/s."""
    out = ctypes.c_double()
    _check(_load().rsos_peak_int(int(kind), int(iters), ctypes.byref(out), _stream(stream)), "rsos_peak_int")
    return out.value


def rsos_checked_build() -> bool:
    """True if the loaded library is the bounds-checked build."""
    return _load().rsos_checked_build() == 1


def rsos_bounds_errors(h, stream=None) -> int:
    """Out-of-range accesses counted for the job (checked build; else 0)."""
    n = ctypes.c_uint32()
    _check(_load().rsos_bounds_errors(h, ctypes.byref(n), _stream(stream)), "rsos_bounds_errors")
    return n.value


def rsos_launches(h) -> int:
    n = ctypes.c_int64()
    _check(_load().rsos_launches(h, ctypes.byref(n)), "rsos_launches")
    return n.value


def rsos_time(h) -> int:
    t = ctypes.c_int64()
    _check(_load().rsos_time(h, ctypes.byref(t)), "rsos_time")
    return t.value


def rsos_free(h) -> None:
    _check(_load().rsos_free(h), "rsos_free")


def rsos_last_cuda_error(h) -> int:
    return int(_load().rsos_last_cuda_error(h))


def rsos_batch_create(params_list, t_max, hbm_budget: int = 0):
    n = len(params_list)
    arr = (rsos_params * n)(*params_list)
    tm = np.ascontiguousarray(t_max, dtype=np.int64)
    b = ctypes.c_void_p()
    _check(_load().rsos_batch_create(arr, _p(tm, ctypes.c_int64), n, int(hbm_budget), ctypes.byref(b)),
           "rsos_batch_create")
    return b


def rsos_batch_schedule(b, job: int, times) -> None:
    a = np.ascontiguousarray(times, dtype=np.int64)
    _check(_load().rsos_batch_schedule(b, int(job), _p(a, ctypes.c_int64), len(a)), "rsos_batch_schedule")


def rsos_batch_run(b, stream=None) -> None:
    rc = _load().rsos_batch_run(b, _stream(stream))
    if rc != RSOS_OK:
        raise RsosError(rc, "rsos_batch_run", _load().rsos_last_cuda_error(None) if rc == RSOS_ECUDA else 0)


def rsos_batch_poll(b, cap: int = 4096):
    """Returns (status, finished job ids); status is RSOS_OK or RSOS_EBUSY."""
    ids = np.zeros(max(cap, 1), dtype=np.int32)
    n = ctypes.c_int32()
    rc = _load().rsos_batch_poll(b, _p(ids, ctypes.c_int32), int(cap), ctypes.byref(n))
    if rc not in (RSOS_OK, RSOS_EBUSY):
        raise RsosError(rc, "rsos_batch_poll", _load().rsos_last_cuda_error(None) if rc == RSOS_ECUDA else 0)
    return rc, [int(v) for v in ids[:n.value]]


def rsos_batch_job(b, job: int):
    h = ctypes.c_void_p()
    _check(_load().rsos_batch_job(b, int(job), ctypes.byref(h)), "rsos_batch_job")
    return h


def rsos_batch_free(b) -> None:
    _check(_load().rsos_batch_free(b), "rsos_batch_free")

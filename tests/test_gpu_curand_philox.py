"""The oracle's Philox-4x32-10 against cuRAND's device implementation of the
same block function (Salmon et al., SC'11), on random and structured
(counter, key) pairs.  The CPU pins fix the Weyl constants by their closed
forms and the statistical quality; this one fixes the multipliers, the round
structure and the word order against an implementation written elsewhere."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("curand") / "curand_philox.so")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", os.path.join(HERE, "host", "curand_philox.cu"), "-o", out])
    lib = ctypes.CDLL(out)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.curand_philox_blocks.argtypes = [u32p, u32p, u32p, ctypes.c_int]
    lib.curand_philox_blocks.restype = ctypes.c_int
    return lib


def _curand(lib, ctr, key):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(ctr)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    rc = lib.curand_philox_blocks(ctr.ctypes.data_as(u32p), key.ctypes.data_as(u32p), out.ctypes.data_as(u32p),
                                  len(ctr))
    assert rc == 0, f"CUDA error {rc}"
    return out


def test_random_pairs(curand_lib):
    rng = np.random.Generator(np.random.PCG64(1605))
    n = 4096
    ctr = rng.integers(0, 1 << 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 1 << 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    got = _curand(curand_lib, ctr, key)
    want = np.stack([O.philox4x32_10(c, k) for c, k in zip(ctr, key)])
    assert np.array_equal(got, want)


def test_counter_layouts_of_the_sweep(curand_lib):
    # the counter shapes the method uses: control (0, t, 0, 1<<30), site
    # (tile, t, g, 2<<30 | p<<28), mask (tile, t, g, 3<<30 | p<<28 | w),
    # including all-zero and all-ones words
    key = np.array([0, 0], dtype=np.uint32)
    ctrs = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [0, 12345, 0, 1 << 30]]
    for tile in (0, 1, 262143):
        for p in range(4):
            ctrs.append([tile, 77, 3, (2 << 30) | (p << 28)])
            ctrs.append([tile, 77, 7, (3 << 30) | (p << 28) | 1])
    ctr = np.array(ctrs, dtype=np.uint32)
    for k in ([0, 0], [1, 0], [0xFFFFFFFF, 0xFFFFFFFF], [123456789, 42]):
        keys = np.tile(np.array(k, dtype=np.uint32), (len(ctr), 1))
        got = _curand(curand_lib, ctr, keys)
        want = np.stack([O.philox4x32_10(c, kk) for c, kk in zip(ctr, keys)])
        assert np.array_equal(got, want), k

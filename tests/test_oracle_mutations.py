"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/rsos_oracle.c (a textual
substitution), compiles the copy on the CPU into a temporary library, and
runs the pins of the affected part against it: the published Philox
known-answer vectors (test_oracle_philox.py) and the hand-built fields of
the constraint checker (test_oracle_max_step.py).  The unmodified source must
pass every pin and every mutant must fail at least one.  Nothing here runs on
a GPU or touches the installed oracle library."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

from test_oracle_max_step import hand_built_cases
from test_oracle_philox import read_kat

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "rsos_oracle.c")

# (name, text to replace, replacement); each must match exactly once
MUTATIONS = [
    ("multipliers swapped", ("#define ORC_PHILOX_M0 0xD2511F53u\n#define ORC_PHILOX_M1 0xCD9E8D57u",
                             "#define ORC_PHILOX_M0 0xCD9E8D57u\n#define ORC_PHILOX_M1 0xD2511F53u")),
    ("Weyl increments swapped", ("#define ORC_PHILOX_W0 0x9E3779B9u", "#define ORC_PHILOX_W0 0xBB67AE85u")),
    ("high and low product words swapped", ("uint32_t y1 = lo1;", "uint32_t y1 = hi1;")),
    ("output words 0 and 2 swapped", ("out[0] = x0; out[1] = x1; out[2] = x2;", "out[0] = x2; out[1] = x1; out[2] = x0;")),
    ("nine rounds", ("for (int round = 0; round < 10; ++round)", "for (int round = 0; round < 9; ++round)")),
    ("key not advanced", ("k0 += ORC_PHILOX_W0;", "k0 += 0u;")),
    ("absolute value dropped along x", ("if (de < 0) de = -de;", "")),
    ("absolute value dropped along y", ("if (ds < 0) ds = -ds;", "")),
    ("vertical pairs ignored", ("if (ds > best) best = ds;", "")),
    ("horizontal wrap ignored", ("int64_t de = v - f[(int64_t)y * L + (x + 1) % L];",
                                 "int64_t de = x + 1 < L ? v - f[(int64_t)y * L + x + 1] : 0;")),
    ("vertical wrap ignored", ("int64_t ds = v - f[(int64_t)((y + 1) % L) * L + x];",
                               "int64_t ds = y + 1 < L ? v - f[(int64_t)(y + 1) * L + x] : 0;")),
]


def build_variant(text: str, tmp: str, name: str):
    c = os.path.join(tmp, name + ".c")
    so = os.path.join(tmp, name + ".so")
    with open(c, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", so, c])
    lib = ctypes.CDLL(so)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
    lib.orc_philox4x32_10.restype = None
    lib.orc_max_step.argtypes = [i64p, ctypes.c_int32, ctypes.c_int32, i64p]
    lib.orc_max_step.restype = None
    return lib


def failed_pins(lib):
    """Names of the pins the library fails."""
    failed = []
    u32p = ctypes.POINTER(ctypes.c_uint32)
    for m, (ctr, key, expected) in enumerate(read_kat()):
        c = np.array(ctr, dtype=np.uint32)
        k = np.array(key, dtype=np.uint32)
        out = np.zeros(4, dtype=np.uint32)
        lib.orc_philox4x32_10(c.ctypes.data_as(u32p), k.ctypes.data_as(u32p), out.ctypes.data_as(u32p))
        if [int(v) for v in out] != expected:
            failed.append(f"philox kat {m}")
    i64p = ctypes.POINTER(ctypes.c_int64)
    for name, field, expected in hand_built_cases():
        f = np.ascontiguousarray(field)
        out = np.zeros(1, dtype=np.int64)
        lib.orc_max_step(f.ctypes.data_as(i64p), f.shape[0], 1, out.ctypes.data_as(i64p))
        if int(out[0]) != expected:
            failed.append(f"max step: {name}")
    return failed


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


def test_unmodified_oracle_passes_every_pin(source, tmp_path):
    assert failed_pins(build_variant(source, str(tmp_path), "original")) == []


@pytest.mark.parametrize("name,sub", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_mutant_fails_a_pin(source, name, sub):
    old, new = sub
    assert source.count(old) == 1, f"mutation site not unique: {old!r}"
    with tempfile.TemporaryDirectory() as tmp:
        lib = build_variant(source.replace(old, new), tmp, "mutant")
        assert failed_pins(lib), f"no pin caught the mutation: {name}"

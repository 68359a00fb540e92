"""Host builds under AddressSanitizer and UndefinedBehaviorSanitizer: the
oracle's dynamics and sums, and the persistent engine's scheduling arithmetic
(the product header compiled for the host), run to completion with no
report.  (compute-sanitizer is not available for the device side; there the
kernels' index arithmetic is covered by the parity tests.)"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
FLAGS = ["-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer"]


def _run(cmd, tmp_path, exe):
    subprocess.check_call(cmd + ["-o", str(tmp_path / exe)])
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([str(tmp_path / exe)], capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "runtime error" not in r.stderr and "AddressSanitizer" not in r.stderr, r.stderr[-3000:]
    return r.stdout.strip()


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_oracle_under_asan_ubsan(tmp_path):
    out = _run(["gcc", "-std=c11", "-fopenmp", *FLAGS, os.path.join(ROOT, "oracle", "rsos_oracle.c"),
                os.path.join(HERE, "host", "oracle_sanitize_main.c")], tmp_path, "oracle_san")
    assert out.isdigit()


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_schedule_arithmetic_under_asan_ubsan(tmp_path):
    out = _run(["g++", "-std=c++17", *FLAGS, "-I", os.path.join(ROOT, "paper_1605_02620_gb300", "csrc"),
                os.path.join(HERE, "host", "sched_sanitize_main.cpp")], tmp_path, "sched_san")
    assert out.isdigit()

"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/rsos.h declares (no compute call is made here)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(rsos_\w+)\s*\(", text, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1605_02620_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert {"rsos_init", "rsos_sweep", "rsos_width", "rsos_free"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_header():
    import paper_1605_02620_gb300 as R
    for n in _declared():
        assert hasattr(R, n), n
    assert R.rsos_strerror(-1) == "invalid argument"


def test_invalid_params_rejected_without_gpu():
    import paper_1605_02620_gb300 as R
    import pytest
    for bad in [R.rsos_params(L=12, N=1, surfaces=64), R.rsos_params(L=64, N=0, surfaces=1),
                R.rsos_params(L=64, N=8, surfaces=1), R.rsos_params(L=64, N=1, surfaces=0),
                R.rsos_params(L=64, N=1, surfaces=1, tile=6)]:
        with pytest.raises(R.RsosError):
            R.rsos_required_bytes(bad)
    assert R.rsos_required_bytes(R.rsos_params(L=4096, N=1, surfaces=64)) >= 2 * 4096 * 4096 * 8


def test_execution_geometry_fields_validated_without_gpu():
    import paper_1605_02620_gb300 as R
    import pytest
    for bad in [dict(surfaces=32, words_per_thread=2),  # one lane word cannot be split in two
                dict(surfaces=64, words_per_thread=3), dict(surfaces=64, tiles_per_lane=65),
                dict(surfaces=64, tiles_per_lane=-1), dict(surfaces=64, phase_lag=1),
                dict(surfaces=64, phase_lag=-2)]:
        with pytest.raises(R.RsosError):
            R.rsos_required_bytes(R.rsos_params(L=256, N=1, **bad))
    for good in [dict(surfaces=64, words_per_thread=1), dict(surfaces=64, words_per_thread=2),
                 dict(surfaces=64, tiles_per_lane=4, phase_lag=12), dict(surfaces=96, words_per_thread=1)]:
        assert R.rsos_required_bytes(R.rsos_params(L=256, N=1, **good)) > 0


def test_restore_rejects_foreign_bytes_without_gpu():
    import paper_1605_02620_gb300 as R
    import pytest
    for junk in (b"", b"RSOSSNP1", b"not a snapshot" * 20, b"RSOSSNP1" + b"\x02\x00\x00\x00" + b"\x00" * 200):
        with pytest.raises(R.RsosError) as e:
            R.rsos_restore(junk)
        assert e.value.status == -1  # RSOS_EINVAL, before any device call


def test_general_tiling_params_validated_without_gpu():
    """(+1) tilings (section III.C): impossible axes, the persistent engine
    where its windows do not fit a block, and single-surface jobs are rejected
    before any device work."""
    import paper_1605_02620_gb300 as R
    import pytest
    ok = dict(L=64, N=1, surfaces=64, tile=(6, 10), tiling=1)
    assert R.rsos_required_bytes(R.rsos_params(**ok)) >= 2 * 64 * 64 * 8
    assert R.rsos_required_bytes(R.rsos_params(L=9605, N=1, surfaces=64, tile=(6, 10), tiling=1)) >= 2 * 9605 ** 2 * 8
    assert R.rsos_required_bytes(R.rsos_params(L=61, N=4, surfaces=64, tile=30, tiling=1)) > 0
    # the persistent engine runs 6(+1) x 10(+1); 30(+1) windows of 4 bit
    # planes are too large for its blocks
    assert R.rsos_required_bytes(R.rsos_params(**dict(ok, engine=2))) > 0
    for bad in [dict(ok, L=10, tile=7), dict(ok, tile=(1, 10)), dict(ok, tile=(6, 31)),
                dict(L=61, N=4, surfaces=64, tile=30, tiling=1, engine=2),
                dict(ok, surfaces=1), dict(ok, tiling=2), dict(ok, L=5, tile=6), dict(ok, N=8)]:
        with pytest.raises(R.RsosError):
            R.rsos_required_bytes(R.rsos_params(**bad))
    # regular tilings keep their rules: 6 x 10 is not a regular tile
    with pytest.raises(R.RsosError):
        R.rsos_required_bytes(R.rsos_params(**dict(ok, tiling=0)))


def test_peak_probe_rejects_bad_arguments_without_gpu():
    import paper_1605_02620_gb300 as R
    import pytest
    for kind, iters in [(3, 10), (-1, 10), (0, 0), (1, -5), (2, 1 << 31)]:
        with pytest.raises(R.RsosError) as e:
            R.rsos_peak_int(kind, iters)
        assert e.value.status == -1


def test_normal_build_is_not_the_checked_one_without_gpu():
    import paper_1605_02620_gb300 as R
    import pytest
    assert R.rsos_checked_build() is False
    with pytest.raises(R.RsosError):
        R.rsos_bounds_errors(None)


def test_wide_word_geometry_validated_without_gpu():
    """128-lane words (words_per_thread = 4) run on the persistent engine with
    8 x 8 tiles and whole 128-lane groups; elsewhere they are rejected before
    any device work."""
    import paper_1605_02620_gb300 as R
    import pytest
    ok = dict(L=256, N=1, surfaces=128, words_per_thread=4)
    for good in [ok, dict(ok, N=7), dict(ok, surfaces=384), dict(ok, engine=2, L=32), dict(ok, surfaces=4096)]:
        assert R.rsos_required_bytes(R.rsos_params(**good)) > 0, good
    for bad in [dict(ok, surfaces=64), dict(ok, surfaces=96), dict(ok, surfaces=160), dict(ok, tile=4, L=64),
                dict(ok, tile=16), dict(ok, engine=1), dict(ok, L=32), dict(ok, surfaces=128 * 33),
                dict(ok, tiling=1, tile=(6, 10)), dict(ok, words_per_thread=3), dict(ok, words_per_thread=5)]:
        with pytest.raises(R.RsosError):
            R.rsos_required_bytes(R.rsos_params(**bad))

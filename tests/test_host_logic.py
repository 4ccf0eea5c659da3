"""Host-side logic that needs no GPU: the autotuner's choice rule and size
buckets, and the tuning table the binding ships and installs (the library's
tuning calls only touch host state)."""
import ctypes
import json

import pytest

from paper_2401_10089_gb300 import _lib


def test_autotune_pick_keeps_configuration_0_on_a_tie():
    pytest.importorskip("torch")
    from paper_2401_10089_gb300.autotune import pick
    assert pick({0: 100.0, 1: 99.0}) == 0          # within the 2 % margin
    assert pick({0: 100.0, 1: 97.0, 2: 98.0}) == 1  # clearly faster
    assert pick({0: 100.0, 3: 101.0}) == 0
    assert pick({1: 50.0, 2: 40.0}) == 2            # no configuration 0 measured


def test_size_buckets_match_the_library():
    pytest.importorskip("torch")
    from paper_2401_10089_gb300.autotune import BUCKET_MAX_N, CANDIDATES, _bucket
    assert [_bucket(n) for n in (1, 8, 9, 16, 17, 32, 33, 64, 65, 128, 129, 256)] == \
        [0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 5, 5]
    assert BUCKET_MAX_N == (8, 16, 32, 64, 128, 256)
    # every candidate configuration can serve its bucket (1: n <= 64, 2 and 4: n <= 32)
    for b, cands in CANDIDATES.items():
        for v in cands:
            assert v in (0, 3) or (v == 1 and b <= 3) or (v in (2, 4) and b <= 2)


def test_shipped_tuning_table_installs_and_bad_tables_are_refused():
    L = _lib.load()
    with open(_lib.TUNING_FILE) as f:
        shipped = json.load(f)["variant"]
    t = _lib.LogmTuning()
    assert L.logm_get_tuning(ctypes.byref(t)) == _lib.SUCCESS
    assert list(t.variant) == shipped  # installed when the library was loaded
    bad = _lib.LogmTuning()
    for i, v in enumerate(shipped):
        bad.variant[i] = v
    bad.variant[5] = 1  # the 128-thread configuration cannot take n <= 256
    assert L.logm_set_tuning(ctypes.byref(bad)) == _lib.ERR_INVALID_ARG
    bad.variant[5] = 7  # no such configuration
    assert L.logm_set_tuning(ctypes.byref(bad)) == _lib.ERR_INVALID_ARG
    assert L.logm_get_tuning(ctypes.byref(t)) == _lib.SUCCESS and list(t.variant) == shipped
    assert L.logm_set_tuning(None) == _lib.SUCCESS  # reset to all-0
    assert L.logm_get_tuning(ctypes.byref(t)) == _lib.SUCCESS and list(t.variant) == [0] * 6
    for i, v in enumerate(shipped):
        t.variant[i] = v
    assert L.logm_set_tuning(ctypes.byref(t)) == _lib.SUCCESS

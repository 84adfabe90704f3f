"""Autotuner host logic on the CPU: cache key, round trip through the
CSVD_TUNE_CACHE file, fallback to an empty cache when the file is missing or
corrupt, the candidate grid, and the library's range checks of the edges."""
import json

import pytest

from paper_2601_11626_gb300 import tune


def test_key_depends_on_shape_not_order():
    a = tune.key("GB300", 2048, [64, 64], [100, 300, 500, 90])
    b = tune.key("GB300", 2048, [64], [500, 90, 300, 100])
    assert a == b
    assert a != tune.key("GB300", 1024, [64], [100, 300, 500, 90])
    assert a != tune.key("GB300", 2048, [32], [100, 300, 500, 90])
    assert a != tune.key("GB300", 2048, [64], [100, 300, 500, 600])


def test_cache_round_trip_and_fallback(tmp_path, monkeypatch):
    path = tmp_path / "tune.json"
    monkeypatch.setenv("CSVD_TUNE_CACHE", str(path))
    assert tune.load_cache() == {}            # missing file
    cache = {"k1": (160, 384), "k2": (192, 320)}
    assert tune.save_cache(cache)
    assert tune.load_cache() == cache
    assert json.loads(path.read_text())["k1"] == [160, 384]
    path.write_text("{not json")
    assert tune.load_cache() == {}            # corrupt file
    path.write_text(json.dumps({"k": [1, 2, 3], "ok": [128, 256]}))
    assert tune.load_cache() == {"ok": (128, 256)}  # malformed entries dropped
    monkeypatch.delenv("CSVD_TUNE_CACHE")
    assert tune.save_cache(cache) is False    # no path: nothing written


def test_candidate_grid_starts_with_default_and_is_ordered():
    c = tune.candidates([100, 200])
    assert c[0] == tune.DEFAULT
    assert all(a < b for a, b in c)
    assert len(set(c)) == len(c)


def test_library_checks_edge_ranges():
    from paper_2601_11626_gb300 import csvd
    lib = csvd.lib(require_gpu=False)
    assert lib.csvd_tune_set(300, 400) == csvd.Status.ERR_ARG   # small edge above 288
    assert lib.csvd_tune_set(200, 150) == csvd.Status.ERR_ARG   # not increasing
    assert lib.csvd_tune_set(160, 384) == 0
    assert tune.get() == (160, 384)
    assert lib.csvd_tune_set(-1, -1) == 0
    assert tune.get() == tune.DEFAULT
    import ctypes
    buf = ctypes.create_string_buffer(512)
    lib.csvd_selftest.argtypes = [ctypes.c_char_p, ctypes.c_int64]
    assert lib.csvd_selftest(buf, 512) == 0, buf.value

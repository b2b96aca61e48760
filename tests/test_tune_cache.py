"""The autotuner's persisted cache (csrc_tune_cache_lookup / csrc_tune_cache_store), host
only: round trips, keys that must not collide, CSRC_TUNE=off, the file location rules, and
lines that do not parse. No GPU is needed."""
import os

import pytest


@pytest.fixture(scope="module")
def cs():
    from paper_1003_0952_gb300 import build

    build.build()
    import paper_1003_0952_gb300 as m

    return m


@pytest.fixture()
def cache(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "dir" / "tune.txt"
    monkeypatch.setenv("CSRC_TUNE_CACHE", str(path))
    monkeypatch.delenv("CSRC_TUNE", raising=False)
    return path


def _key(cs, h=0x1234ABCD5678EF01, n=1000, nnz=6000, storage=0, flags=0, device=b"NVIDIA GB300/152SM"):
    k = cs.csrc_tune_key()
    k.pattern_hash, k.n, k.nnz, k.storage, k.flags, k.device = h, n, nnz, storage, flags, device
    return k


def test_round_trip_and_replacement(cs, cache):
    k = _key(cs)
    assert cs.csrc_tune_cache_lookup(k, cs.CSRC_TUNE_STRATEGY) is None
    cs.csrc_tune_cache_store(k, cs.CSRC_TUNE_STRATEGY, 0.0, [1, 2432])
    assert cache.exists()  # directories are created
    assert cs.csrc_tune_cache_lookup(k, cs.CSRC_TUNE_STRATEGY) == [1, 2432, 0, 0]
    cs.csrc_tune_cache_store(k, cs.CSRC_TUNE_STRATEGY, 0.0, [3, 608])
    assert cs.csrc_tune_cache_lookup(k, cs.CSRC_TUNE_STRATEGY) == [3, 608, 0, 0]
    assert len(cache.read_text().splitlines()) == 1  # replaced, not appended


def test_keys_do_not_collide(cs, cache):
    base = dict(h=7, n=10, nnz=28, storage=0, flags=0, device=b"dev A")
    variants = [dict(base, h=8), dict(base, n=11), dict(base, nnz=29), dict(base, storage=1),
                dict(base, flags=16), dict(base, device=b"dev B")]
    cs.csrc_tune_cache_store(_key(cs, **base), cs.CSRC_TUNE_STRATEGY, 0.0, [1, 5])
    for i, v in enumerate(variants):
        assert cs.csrc_tune_cache_lookup(_key(cs, **v), cs.CSRC_TUNE_STRATEGY) is None
        cs.csrc_tune_cache_store(_key(cs, **v), cs.CSRC_TUNE_STRATEGY, 0.0, [2, 100 + i])
    assert cs.csrc_tune_cache_lookup(_key(cs, **base), cs.CSRC_TUNE_STRATEGY) == [1, 5, 0, 0]
    for i, v in enumerate(variants):
        assert cs.csrc_tune_cache_lookup(_key(cs, **v), cs.CSRC_TUNE_STRATEGY) == [2, 100 + i, 0, 0]
    # kinds and parameters are part of the key as well
    k = _key(cs, **base)
    cs.csrc_tune_cache_store(k, cs.CSRC_TUNE_KTILE, 8.0, [4])
    cs.csrc_tune_cache_store(k, cs.CSRC_TUNE_KTILE, 32.0, [8])
    cs.csrc_tune_cache_store(k, cs.CSRC_TUNE_PRECISION, 1e-5, [1])
    cs.csrc_tune_cache_store(k, cs.CSRC_TUNE_PRECISION, 1e-12, [0])
    assert cs.csrc_tune_cache_lookup(k, cs.CSRC_TUNE_KTILE, 8.0)[0] == 4
    assert cs.csrc_tune_cache_lookup(k, cs.CSRC_TUNE_KTILE, 32.0)[0] == 8
    assert cs.csrc_tune_cache_lookup(k, cs.CSRC_TUNE_KTILE, 16.0) is None
    assert cs.csrc_tune_cache_lookup(k, cs.CSRC_TUNE_PRECISION, 1e-5)[0] == 1
    assert cs.csrc_tune_cache_lookup(k, cs.CSRC_TUNE_PRECISION, 1e-12)[0] == 0


def test_off_mode_reads_and_writes_nothing(cs, cache, monkeypatch):
    k = _key(cs)
    cs.csrc_tune_cache_store(k, cs.CSRC_TUNE_STRATEGY, 0.0, [1, 9])
    before = cache.read_text()
    monkeypatch.setenv("CSRC_TUNE", "off")
    assert cs.csrc_tune_cache_lookup(k, cs.CSRC_TUNE_STRATEGY) is None
    cs.csrc_tune_cache_store(k, cs.CSRC_TUNE_STRATEGY, 0.0, [2, 10])
    assert cache.read_text() == before
    monkeypatch.setenv("CSRC_TUNE", "full")  # full still records and looks up
    assert cs.csrc_tune_cache_lookup(k, cs.CSRC_TUNE_STRATEGY) == [1, 9, 0, 0]


def test_unparsable_lines_are_ignored_and_dropped(cs, cache):
    k = _key(cs)
    cache.parent.mkdir(parents=True, exist_ok=True)
    cache.write_text("garbage line\n\ncsrc-tune-v1 not enough fields\n")
    assert cs.csrc_tune_cache_lookup(k, cs.CSRC_TUNE_STRATEGY) is None
    cs.csrc_tune_cache_store(k, cs.CSRC_TUNE_STRATEGY, 0.0, [1, 3])
    assert cs.csrc_tune_cache_lookup(k, cs.CSRC_TUNE_STRATEGY) == [1, 3, 0, 0]
    assert "garbage" not in cache.read_text()


def test_default_location(cs, tmp_path, monkeypatch):
    monkeypatch.delenv("CSRC_TUNE_CACHE", raising=False)
    monkeypatch.delenv("CSRC_TUNE", raising=False)
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path / "xdg"))
    k = _key(cs, h=99)
    cs.csrc_tune_cache_store(k, cs.CSRC_TUNE_STRATEGY, 0.0, [1, 1])
    assert (tmp_path / "xdg" / "csrc_gb300" / "tune.txt").exists()
    monkeypatch.delenv("XDG_CACHE_HOME")
    monkeypatch.setenv("HOME", str(tmp_path / "home"))
    cs.csrc_tune_cache_store(k, cs.CSRC_TUNE_STRATEGY, 0.0, [1, 2])
    assert (tmp_path / "home" / ".cache" / "csrc_gb300" / "tune.txt").exists()


def test_invalid_arguments(cs, cache):
    import ctypes

    k = _key(cs)
    v = (ctypes.c_int32 * 4)()
    lib = cs.lib()
    assert lib.csrc_tune_cache_lookup(None, 0, 0.0, v) == cs.CSRC_ERR_INVALID_ARG
    assert lib.csrc_tune_cache_lookup(ctypes.byref(k), 7, 0.0, v) == cs.CSRC_ERR_INVALID_ARG
    assert lib.csrc_tune_cache_store(ctypes.byref(k), 0, float("nan"), v) == cs.CSRC_ERR_INVALID_ARG
    assert lib.csrc_get_tune_key(None, ctypes.byref(k)) == cs.CSRC_ERR_INVALID_ARG

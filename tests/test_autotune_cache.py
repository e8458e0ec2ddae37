"""The autotuner's JSON cache, on the CPU: the library's variant registry
needs no device, and the GPU-name part of the cache key is replaced."""
import json

import pytest

from paper_2203_09384_gb300 import _abi, autotune

KEY = "GB300 (test)"


@pytest.fixture
def fake_gpu(monkeypatch):
    monkeypatch.setattr(autotune, "_device_key",
                        lambda device=None: f"{KEY}|{autotune.schedule_fingerprint()}")
    saved = {n: _abi.fft_get_default_variant(n) for n in autotune.LENGTHS}
    saved_ragged = _abi.fft_get_default_ragged_variant()
    yield
    for n, v in saved.items():
        _abi.fft_set_default_variant(n, v)
    _abi.fft_set_default_ragged_variant(saved_ragged)


def fp32_variants(n):
    return [v for v in range(_abi.fft_variant_count(n)) if _abi.fft_variant_dtype(n, v) == _abi.FFT_C64]


def test_round_trip_applies_the_tuned_defaults(fake_gpu, tmp_path):
    n = next(n for n in autotune.LENGTHS if len(fp32_variants(n)) > 1)
    other = fp32_variants(n)[-1]
    assert other != _abi.fft_get_default_variant(n)
    path = str(tmp_path / "tune.json")
    autotune.save_cache({n: {"best": other, "ms": {}}}, {"best": 6, "ms": {}}, path=path)
    entry = autotune.load_cache(path=path)
    assert entry["plain"] == {str(n): other} and entry["ragged"] == 6
    assert _abi.fft_get_default_variant(n) == other


def test_cached_ragged_variant_becomes_the_default(fake_gpu, tmp_path):
    """The tuner's ragged choice is applied through
    fft_set_default_ragged_variant, so later ragged plans that name no variant
    start from it; a value outside the compiled variants is ignored."""
    count = _abi.fft_ragged_variant_count()
    want = next(v for v in range(count) if v != _abi.fft_get_default_ragged_variant())
    path = str(tmp_path / "tune.json")
    autotune.save_cache(None, {"best": want, "ms": {}}, path=path)
    assert autotune.load_cache(path=path)["ragged"] == want
    assert _abi.fft_get_default_ragged_variant() == want
    key = autotune._device_key()
    for bad in (count, -1, "6"):
        (tmp_path / "bad.json").write_text(json.dumps({key: {"ragged": bad}}))
        autotune.load_cache(path=str(tmp_path / "bad.json"))
        assert _abi.fft_get_default_ragged_variant() == want
    with pytest.raises(_abi.FFTError):
        _abi.fft_set_default_ragged_variant(count)


def test_autoload_applies_the_cache_once(fake_gpu, tmp_path, monkeypatch):
    """Plans call autotune.autoload() before their first creation: the cache
    at GBFFT_TUNE_CACHE is applied once per process, and "off" disables it."""
    want = (_abi.fft_get_default_ragged_variant() + 1) % _abi.fft_ragged_variant_count()
    path = str(tmp_path / "tune.json")
    autotune.save_cache(None, {"best": want, "ms": {}}, path=path)
    monkeypatch.setenv("GBFFT_TUNE_CACHE", path)
    monkeypatch.setattr(autotune, "_autoload_done", False)
    autotune.autoload()
    assert _abi.fft_get_default_ragged_variant() == want
    _abi.fft_set_default_ragged_variant((want + 1) % _abi.fft_ragged_variant_count())
    autotune.autoload()  # already done in this process: no second application
    assert _abi.fft_get_default_ragged_variant() != want
    monkeypatch.setenv("GBFFT_TUNE_CACHE", "off")
    monkeypatch.setattr(autotune, "_autoload_done", False)
    autotune.autoload()
    assert _abi.fft_get_default_ragged_variant() != want


def test_entries_that_cannot_be_defaults_are_skipped(fake_gpu, tmp_path):
    n = next(n for n in autotune.LENGTHS
             if any(_abi.fft_variant_dtype(n, v) != _abi.FFT_C64 for v in range(_abi.fft_variant_count(n))))
    not_fp32 = next(v for v in range(_abi.fft_variant_count(n)) if _abi.fft_variant_dtype(n, v) != _abi.FFT_C64)
    before = _abi.fft_get_default_variant(n)
    path = tmp_path / "tune.json"
    key = autotune._device_key()
    path.write_text(json.dumps({key: {"plain": {str(n): not_fp32, "64": 99, "2": -1}}}))
    autotune.load_cache(path=str(path))
    assert _abi.fft_get_default_variant(n) == before


def test_other_tables_and_broken_files_are_ignored(fake_gpu, tmp_path):
    path = tmp_path / "tune.json"
    n = next(n for n in autotune.LENGTHS if len(fp32_variants(n)) > 1)
    before = _abi.fft_get_default_variant(n)
    stale = f"{KEY}|an older variant table"
    path.write_text(json.dumps({stale: {"plain": {str(n): fp32_variants(n)[-1]}}}))
    assert autotune.load_cache(path=str(path)) == {}
    assert _abi.fft_get_default_variant(n) == before
    path.write_text("{not json")
    assert autotune.load_cache(path=str(path)) == {}
    assert autotune.load_cache(path=str(tmp_path / "missing.json")) == {}


def test_fingerprint_names_every_length():
    fp = autotune.schedule_fingerprint()
    assert all(f"{n}:" in fp for n in autotune.LENGTHS)
    assert fp.endswith(f";r{_abi.fft_ragged_variant_count()}")

"""Host logic of the batched kernel's autotuner, without a GPU: the input-mix
key that choices are cached under, and the cache itself (first use tunes and
stores, later uses read the stored choice, a retune replaces it, and a
missing or corrupt cache file is treated as empty)."""
import json
from types import SimpleNamespace

import pytest

from paper_2109_10433_gb300 import autotune as T


def batch(units, count):
    return SimpleNamespace(units=units, count=count)


def test_mix_key_buckets():
    # all UTF-8, all UTF-16 (2 bytes a unit), and an even split by bytes
    assert T.mix_key(batch(1 << 20, 1024), None) == "share16=0|size=2^20|mean=2^10"
    assert T.mix_key(None, batch(1 << 19, 1024)) == "share16=4|size=2^20|mean=2^10"
    assert T.mix_key(batch(1 << 19, 512), batch(1 << 18, 512)) == "share16=2|size=2^20|mean=2^10"
    # sizes within one power of two share a key; the next power does not
    assert T.mix_key(batch(1_500_000, 1000), None) == T.mix_key(batch(1_100_000, 1000), None)
    assert T.mix_key(batch(1 << 21, 1000), None) != T.mix_key(batch(1 << 20, 1000), None)
    # empty batches
    assert T.mix_key(None, None) == "share16=0|size=2^0|mean=2^0"
    assert T.mix_key(batch(0, 0), batch(0, 0)) == "share16=0|size=2^0|mean=2^0"


def test_cache_tunes_once_then_reads(tmp_path, monkeypatch):
    path = tmp_path / "cache.json"
    monkeypatch.setattr(T, "CACHE_PATH", str(path))
    monkeypatch.setattr(T, "_device_key", lambda: "GB300|152|13.0")
    calls = []

    def fake_tune(b8, b16, ws, reps=5):
        calls.append(reps)
        times = {0: 3.0, 1: 1.5, 2: 2.0, 3: 4.0}
        return min(times, key=times.get), times

    monkeypatch.setattr(T, "tune", fake_tune)
    b8, b16 = batch(1 << 20, 1000), batch(1 << 19, 1000)
    assert T.best_config(b8, b16, ws=None) == 1
    assert T.best_config(b8, b16, ws=None) == 1
    assert len(calls) == 1                          # the second call read the cache
    stored = json.loads(path.read_text())
    key = "GB300|152|13.0|" + T.mix_key(b8, b16)
    assert stored[key]["config"] == 1 and stored[key]["ms"]["1"] == 1.5
    # another mix tunes again; a retune replaces the stored choice
    assert T.best_config(batch(1 << 10, 4), None, ws=None) == 1
    assert len(calls) == 2
    monkeypatch.setattr(T, "tune", lambda *a, **k: (3, {3: 0.5}))
    assert T.best_config(b8, b16, ws=None) == 1
    assert T.best_config(b8, b16, ws=None, retune=True) == 3
    assert T.best_config(b8, b16, ws=None) == 3
    assert len(json.loads(path.read_text())) == 2


def test_missing_or_corrupt_cache_reads_as_empty(tmp_path, monkeypatch):
    path = tmp_path / "cache.json"
    monkeypatch.setattr(T, "CACHE_PATH", str(path))
    assert T._load() == {}
    path.write_text("{not json")
    assert T._load() == {}
    T._store({"k": {"config": 2}})
    assert T._load() == {"k": {"config": 2}}
    assert not list(tmp_path.glob("*.tmp*"))       # written through a temporary file, renamed


@pytest.mark.parametrize("share", [0, 1, 2, 3, 4])
def test_share_of_utf16_bytes_in_quarters(share):
    total = 1 << 20
    u16_bytes = total * share // 4
    b8 = batch(total - u16_bytes, 10) if total - u16_bytes else None
    b16 = batch(u16_bytes // 2, 10) if u16_bytes else None
    assert T.mix_key(b8, b16).startswith(f"share16={share}|")

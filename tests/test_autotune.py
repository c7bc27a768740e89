"""Host logic of the autotuner: the search over candidates and the persistent cache (no GPU: the timing and the
context are fakes)."""
import importlib
import json

T = importlib.import_module("paper_2407_19151_gb300.autotune")  # the package attribute is the function


def test_search_keeps_fastest_and_skips_duplicates():
    applied, timed = [], []
    times = {0: 5.0, 128: 3.0, 160: 3.0, 192: 4.0, 256: None}  # 128 and 160 give the same capacities

    def apply(c):
        applied.append(c)
        return 128 if c in (128, 160) else c

    def time_one():
        timed.append(applied[-1])
        return times[applied[-1]]

    best, ms = T.search((0, 128, 160, 192, 256), apply, time_one)
    assert best == 128 and ms == 3.0
    assert timed == [0, 128, 192, 256]       # 160 coincides with 128; 256 failed and is not chosen
    assert applied[-1] == 128                # the winner is applied last


def test_search_all_failed_applies_first():
    applied = []
    best, ms = T.search((0, 64), lambda c: applied.append(c) or c, lambda: None)
    assert best == 0 and applied[-1] == 0


def test_cache_round_trip(tmp_path, monkeypatch):
    path = tmp_path / "sub" / "autotune.json"
    monkeypatch.setenv("MCC_AUTOTUNE_CACHE", str(path))
    assert T.cache_path() == str(path)
    k1 = T.cache_key("GB300", 152, "f32", False, 1 << 18, 134_296_981, 4733, "abc")
    k2 = T.cache_key("GB300", 152, "f32", True, 1 << 18, 134_296_981, 4733, "abc")
    assert k1 != k2
    T._store(str(path), k1, {"group_cap": 0, "tile_cap": 0, "ms": 1.0})
    T._store(str(path), k2, {"group_cap": 192, "tile_cap": 512, "ms": 2.0})
    d = json.loads(path.read_text())
    assert d[k1]["group_cap"] == 0 and d[k2]["tile_cap"] == 512
    assert T._load(str(tmp_path / "missing.json")) == {}
    path.write_text("not json")
    assert T._load(str(path)) == {}

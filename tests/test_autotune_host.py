"""Host logic of the autotuner (no GPU): workload signatures, the JSON cache
round trip, and the rule that a cached choice is used only while every value
in it is still one of the current candidates (the tile selector values follow
the compiled tile variants, so an entry written for other variants is tuned
again rather than applied)."""
from paper_1704_08579_gb300 import autotune


def test_signature_buckets_sizes_by_power_of_two():
    assert autotune.signature("i32", 530_045_367, 20_000) == "i32:n2^28:seg2^14"
    assert autotune.signature("f64", 1 << 28, 1) == "f64:n2^28:seg2^0"
    assert autotune.signature("kv", 0, 0) == "kv:n2^0:seg2^0"


def test_cache_round_trip(tmp_path, monkeypatch):
    monkeypatch.setattr(autotune, "CACHE_DIR", str(tmp_path))
    assert autotune._load_cache("NVIDIA GB300") == {}
    entry = {"leaf_max": 16384, "small_max": 512, "driver_items": autotune.ITEMS_CHOICES["f64"][0], "ms": 1.5}
    autotune._store_cache("NVIDIA GB300", {"f64:n2^20:seg2^3": entry})
    assert autotune._load_cache("NVIDIA GB300") == {"f64:n2^20:seg2^3": entry}
    assert [p.name for p in tmp_path.iterdir()] == ["NVIDIA_GB300.json"]


def test_cached_entry_accepts_only_current_candidates():
    for kind in ("i32", "f64", "kv"):
        good = {"leaf_max": autotune.LEAF_CHOICES[kind][0], "small_max": autotune.SMALL_CHOICES[-1],
                "driver_items": autotune.ITEMS_CHOICES[kind][0], "ms": 2.0}
        cache = {"s": good}
        assert autotune.cached_entry(cache, "s", kind) is good
        assert autotune.cached_entry(cache, "other", kind) is None
        for key, bad in (("driver_items", 64), ("leaf_max", 3), ("small_max", 1000)):
            assert autotune.cached_entry({"s": dict(good, **{key: bad})}, "s", kind) is None
    # The register tile of FP64 / key/value sorts was once selected by 32: such an entry is stale now.
    stale = {"leaf_max": 16384, "small_max": 512, "driver_items": 32, "ms": 1.0}
    if 32 not in autotune.ITEMS_CHOICES["f64"]:
        assert autotune.cached_entry({"s": stale}, "s", "f64") is None
    assert autotune.cached_entry({"s": "garbage"}, "s", "i32") is None

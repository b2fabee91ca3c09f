"""Host logic of the autotuner's JSON cache layer: cache keys, lookup, store, re-tune (no GPU)."""
import json

from paper_2302_12727_gb300 import autotune as A


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "cache.json")
    calls, applied = [], []

    def tune():
        calls.append(1)
        return {"flux_variant": 2, "gather_variant": 1, "gradient_variant": 0}, [1.0] * 18

    key = A.shape_key(1000, 3, 24000, "glf", "fp32")
    e1 = A.lookup_or_tune(key, tune, applied.append, path)
    assert e1["source"] == "measured" and len(calls) == 1
    e2 = A.lookup_or_tune(key, tune, applied.append, path)
    assert e2["source"] == "cache" and len(calls) == 1
    assert applied == [e1["tuning"], e1["tuning"]]
    # another shape misses; re-tune measures again
    A.lookup_or_tune(A.shape_key(1000, 4, 24000, "glf", "fp32"), tune, applied.append, path)
    A.lookup_or_tune(key, tune, applied.append, path, retune=True)
    assert len(calls) == 3
    data = json.load(open(path))
    assert set(data) == {key, A.shape_key(1000, 4, 24000, "glf", "fp32")}


def test_unreadable_cache_is_ignored(tmp_path):
    path = tmp_path / "cache.json"
    path.write_text("{not json")
    assert A.load_cache(str(path)) == {}
    e = A.lookup_or_tune("k", lambda: ({"flux_variant": 0, "gather_variant": 0, "gradient_variant": 0}, []),
                         lambda t: None, str(path))
    assert e["source"] == "measured" and json.load(open(path))["k"]["tuning"]["flux_variant"] == 0

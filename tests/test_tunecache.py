"""Host logic of the autotuner cache (no GPU): keys, storage, and that a cache
hit sets the stored knobs without timing anything."""

import json

import pytest

from paper_2401_12501_gb300 import tunecache


def test_size_bucket_is_nearest_power_of_two_in_log_scale():
    assert tunecache.size_bucket(1) == 1
    assert tunecache.size_bucket(9600) == 8192        # log2 9600 = 13.23
    assert tunecache.size_bucket(12000) == 16384      # log2 12000 = 13.55
    assert tunecache.size_bucket(98304) == 131072     # log2 98304 = 16.58
    assert tunecache.size_bucket(65536) == 65536
    with pytest.raises(ValueError):
        tunecache.size_bucket(0)


def test_key_names_gpu_bucket_nrhs_and_precision():
    assert tunecache.tune_key("NVIDIA GB300", 24576, 64, "fp32") == "NVIDIA GB300|N~32768|nrhs=64|fp32"
    assert tunecache.tune_key("g", 9000, 1, "fmm") == tunecache.tune_key("g", 9600, 1, "fmm")
    assert tunecache.tune_key("g", 9600, 1, "fmm") != tunecache.tune_key("g", 9600, 2, "fmm")


def entry(**kn):
    k = {f: 0 for f in tunecache.KNOB_FIELDS}
    k.update(kn)
    return {"knobs": k, "best_ms": 0.05, "default_ms": 0.06, "candidates": 13, "N": 9600}


def test_store_and_load_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    assert tunecache.load(path) == {}
    tunecache.store(path, "a", entry(direct_tpt=4))
    tunecache.store(path, "b", entry(batch_rhs_per_block=32))
    tunecache.store(path, "a", entry(direct_tpt=1))           # replaces
    data = tunecache.load(path)
    assert set(data) == {"a", "b"}
    assert data["a"]["knobs"]["direct_tpt"] == 1
    assert data["b"]["knobs"]["batch_rhs_per_block"] == 32
    assert not [p for p in tmp_path.iterdir() if p.name.startswith(".tunecache")]


def test_invalid_entries_and_corrupt_files(tmp_path):
    path = str(tmp_path / "tune.json")
    with pytest.raises(ValueError):
        tunecache.store(path, "a", {"knobs": {"direct_tpt": 1}})
    with pytest.raises(ValueError):
        tunecache.store(path, "a", entry(direct_tpt=1.5))
    (tmp_path / "tune.json").write_text("{not json")
    assert tunecache.load(path) == {}
    tunecache.store(path, "a", entry())
    assert json.loads((tmp_path / "tune.json").read_text())["a"]["N"] == 9600


def test_cache_hit_sets_knobs_without_timing(tmp_path, monkeypatch):
    import paper_2401_12501_gb300 as pm

    class FakeCtx:
        def info(self):
            return "FAKE GPU", 152

    s = object.__new__(pm.Surface)
    s.ctx, s.N, s.handle = FakeCtx(), 9600, None
    seen = {}
    monkeypatch.setattr(pm.Surface, "set_knobs", lambda self, **kw: seen.update(kw))
    path = str(tmp_path / "tune.json")
    key = tunecache.tune_key("FAKE GPU", 9600, 1, "fp32")
    tunecache.store(path, key, entry(direct_tpt=4, direct_blocks_per_sm=8))
    r = s.autotune(nrhs=1, prec="fp32", cache=path)
    assert r["cached"] and r["key"] == key
    assert seen["direct_tpt"] == 4 and seen["direct_blocks_per_sm"] == 8

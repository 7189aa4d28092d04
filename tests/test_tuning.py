"""The option autotuner's host logic: shape keys, cache lookup (exact,
nearest row count, default) and recording of measured candidates.  No GPU:
the cache here is written by the test."""
import json

from paper_2010_00152_gb300 import tuning


def test_shape_key_buckets():
    assert tuning.shape_key("batched", 2_072_320_040, 32, 4, 0.975) == "batched|n30|k32|s4|d3"
    assert tuning.shape_key("aggregate", 1 << 29, 64, 2, 0.5676) == "aggregate|n29|k64|s2|d2"
    assert tuning.shape_key("aggregate", (1 << 20) + 5, 64, 4, 0.0) == "aggregate|n20|k64|s4|d0"
    assert tuning.shape_key("aggregate", 1000, 16, 1, None) == "aggregate|n9|k16|s1"
    assert [tuning.dup_bucket(x) for x in (0.0, 0.0999, 0.1, 0.4999, 0.5, 0.8999, 0.9, 1.0)] == \
        [0, 0, 1, 1, 2, 2, 3, 3]


def test_record_keeps_the_fastest_and_every_time(tmp_path):
    cache = {}
    best = tuning.record(cache, "batched|n30|k32|s4|d3",
                         [({}, 154.5), ({"batch_group_rows": 1 << 28}, 124.8), ({"batch_group_rows": 1 << 27}, 130.3)],
                         "test")
    assert best == {"batch_group_rows": 1 << 28}
    e = cache["batched|n30|k32|s4|d3"]
    assert e["best"] == best and len(e["ms"]) == 3 and e["ms"]["{}"] == 154.5
    p = tmp_path / "t.json"
    tuning.save(cache, str(p))
    assert tuning.load(str(p)) == json.loads(p.read_text())


def test_choose_exact_nearest_default():
    cache = {}
    tuning.record(cache, "batched|n30|k32|s4|d3", [({"batch_group_rows": 1 << 28}, 1.0)], "t")
    tuning.record(cache, "batched|n26|k32|s4|d3", [({"batch_group_rows": 1 << 25}, 1.0)], "t")
    tuning.record(cache, "aggregate|n29|k64|s2|d2", [({"merge_copy": 2}, 1.0)], "t")
    assert tuning.choose("batched|n30|k32|s4|d3", cache) == ({"batch_group_rows": 1 << 28}, "cache",
                                                             "batched|n30|k32|s4|d3")
    # nearest row count of the same call, key bits, aggregates and duplicates
    assert tuning.choose("batched|n27|k32|s4|d3", cache)[0] == {"batch_group_rows": 1 << 25}
    assert tuning.choose("batched|n29|k32|s4|d3", cache)[1:] == ("nearest", "batched|n30|k32|s4|d3")
    # no duplicate bucket given: any bucket of the same kind matches
    assert tuning.choose("batched|n31|k32|s4", cache)[0] == {"batch_group_rows": 1 << 28}
    # another call, key width, aggregate count or duplicate bucket: the defaults
    for k in ("served|n30|k32|s4|d3", "batched|n30|k64|s4|d3", "batched|n30|k32|s2|d3", "batched|n30|k32|s4|d1"):
        assert tuning.choose(k, cache) == ({}, "default", None)


def test_shipped_cache_is_well_formed():
    """The cache that ships with the package: every entry names its best
    option set among its measured candidates, and only known options."""
    known = {"prefold", "radix_bits", "fanin_cap", "merge_copy", "prefold_bins", "prefold_rows", "one_pass",
             "part_levels", "batch_group_rows", "lowcard", "merge_threads"}
    cache = tuning.load()
    for key, e in cache.items():
        f = key.split("|")
        assert f[0] in ("batched", "aggregate") and all(x[0] in "nksd" for x in f[1:])
        assert json.dumps(e["best"], sort_keys=True) in e["ms"]
        assert e["ms"][json.dumps(e["best"], sort_keys=True)] == min(e["ms"].values())
        assert set(e["best"]) <= known

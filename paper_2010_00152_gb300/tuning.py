"""Option autotuner: library options for a call shape, from a JSON cache of
timings measured on the GPU.

Every option it sets leaves the result unchanged (run generation, merge
and partitioning knobs only); it changes how fast a call runs.  A shape is

    <call>|n<floor(log2 rows)>|k<key bits>|s<aggregates>|d<duplicate bucket>

where the duplicate bucket is the share of input rows that fold into
another row (1 - output rows / input rows): d0 below 0.1, d1 below 0.5, d2
below 0.9, d3 from 0.9 up.  Callers that know the rate from an earlier call
on the same data (a served or repeated workload) pass it; otherwise d is
left out of the match.

The cache (tuning.json beside this file) maps a shape to the option set that
measured fastest and to every candidate's time:

    {"batched|n30|k32|s4|d3": {"best": {"batch_group_rows": 268435456},
                               "ms": {"{}": 154.5, ...},
                               "measured": "GB300, 3 calls after 1 warm-up"}}

`bench.py --tune` measures candidate sets and writes the entries.  A shape
missing from the cache takes the entry of the same call, key bits,
aggregates and duplicate bucket with the nearest row count, else the
library defaults.
"""
import json
import math
import os

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def dup_bucket(dup):
    """Bucket of a duplicate share in [0, 1]."""
    if dup is None:
        return None
    return 0 if dup < 0.1 else (1 if dup < 0.5 else (2 if dup < 0.9 else 3))


def shape_key(call, n_rows, key_bits, n_aggs, dup=None):
    nb = int(math.floor(math.log2(n_rows))) if n_rows > 0 else 0
    key = "%s|n%d|k%d|s%d" % (call, nb, key_bits, n_aggs)
    d = dup_bucket(dup)
    return key if d is None else key + "|d%d" % d


def _parse(key):
    parts = key.split("|")
    f = {"call": parts[0]}
    for p in parts[1:]:
        f[p[0]] = int(p[1:])
    return f


def load(path=CACHE):
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        return json.load(fh)


def choose(key, cache=None):
    """(options, source, matched key): source is "cache" for the shape
    itself, "nearest" for the nearest row count of the same kind of call,
    "default" when nothing matches (empty options)."""
    cache = load() if cache is None else cache
    if key in cache:
        return dict(cache[key]["best"]), "cache", key
    want = _parse(key)
    best, best_d = None, None
    for k in cache:
        f = _parse(k)
        if f["call"] != want["call"] or f.get("k") != want.get("k") or f.get("s") != want.get("s"):
            continue
        if "d" in want and f.get("d") != want["d"]:
            continue
        dist = abs(f.get("n", 0) - want.get("n", 0))
        if best_d is None or dist < best_d or (dist == best_d and k < best):
            best, best_d = k, dist
    if best is None:
        return {}, "default", None
    return dict(cache[best]["best"]), "nearest", best


def record(cache, key, timings, note):
    """Store the candidates' times (option dict -> ms) under key, the fastest
    as its best; returns the best option set."""
    items = sorted(timings, key=lambda t: t[1])
    cache[key] = {"best": dict(items[0][0]),
                  "ms": {json.dumps(o, sort_keys=True): round(ms, 3) for o, ms in timings},
                  "measured": note}
    return dict(items[0][0])


def save(cache, path=CACHE):
    with open(path, "w") as fh:
        json.dump(cache, fh, indent=1, sort_keys=True)
        fh.write("\n")

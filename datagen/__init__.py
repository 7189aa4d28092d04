"""Seeded synthetic inputs for the grouping workloads.

Holds none of the grouping method's arithmetic: only counter-based random
numbers and the recipes that shape them into key and payload columns.  Both
the oracle-side tests and the CUDA path draw their inputs from here; every
function gives identical values on the CPU and on a CUDA device because it
uses only wrapping int64 arithmetic in torch.

Generators (published definitions, restated):
  * SplitMix64 finalizer (Steele, Lea, Flood, "Fast splittable pseudorandom
    number generators", OOPSLA 2014) -- a bijection on 64-bit words, used both
    as a counter-based RNG (mix64(base + i)) and to spread key indices over
    the whole 64-bit key space.
  * MurmurHash3 fmix32 finalizer (Appleby) -- a bijection on 32-bit words,
    for uint32 keys.

Workloads (sizes use binary prefixes; see the design notes for the recipe):
  c1  n=2^20, uint64 keys = mix64(U[0,10^4)), payload U[-1000,1000],
      count/sum/min/max, memory budget 65,536 rows.
  c2  n=2^28, two uint8 key columns with 4 combinations at 49/25/24/2 %,
      four payload columns U[0,10^7), count + sum/min/max per column.
  c3  n=2^29, uint64 keys = mix64(U[0,2^28)), payload U[-10^9,10^9],
      count/sum, memory budget 2^25 rows.
  c4  4,096 instances, rows log-uniform [2^10,2^22], uint32 keys =
      fmix32(Zipf(1.1) rank over a domain log-uniform [16,2^20]),
      payload U[-1000,1000], count/sum/min/max.
  c5  request stream: rows log-uniform [2^10,2^24], distinct/rows
      log-uniform [0.001,1], uint64 keys, payloads U[-1000,1000] and
      U[0,10^7), count + sum/min/max of both.
"""
import math

import numpy as np
import torch

MASK64 = (1 << 64) - 1


def _s64(c):
    """A 64-bit constant as the int64 with the same bits."""
    c &= MASK64
    return c - (1 << 64) if c >= (1 << 63) else c


_GOLDEN = _s64(0x9E3779B97F4A7C15)
_M1 = _s64(0xBF58476D1CE4E5B9)
_M2 = _s64(0x94D049BB133111EB)


def _shr(x, k):
    """Logical right shift of int64 tensors (torch shifts arithmetically)."""
    return (x >> k) & ((1 << (64 - k)) - 1)


def mix64(x):
    """SplitMix64 finalizer on an int64 tensor (bit pattern of a uint64)."""
    z = x + _GOLDEN
    z = (z ^ _shr(z, 30)) * _M1
    z = (z ^ _shr(z, 27)) * _M2
    return z ^ _shr(z, 31)


def fmix32(x):
    """MurmurHash3 32-bit finalizer on int64 tensors holding uint32 values."""
    m = 0xFFFFFFFF
    h = x & m
    h = h ^ (h >> 16)
    h = (h * 0x85EBCA6B) & m
    h = h ^ (h >> 13)
    h = (h * 0xC2B2AE35) & m
    h = h ^ (h >> 16)
    return h


def stream_base(seed, stream):
    """Start of an independent counter stream for (seed, stream)."""
    t = torch.tensor([_s64(seed * 0x100000001B3 + stream * 0x9E3779B1)], dtype=torch.int64)
    return int(mix64(mix64(t))[0])


def rand64(seed, stream, n, device="cpu", start=0):
    """n pseudo-random 64-bit words (as int64) of stream (seed, stream)."""
    base = stream_base(seed, stream)
    i = torch.arange(start, start + n, dtype=torch.int64, device=device)
    return mix64(i + base)


def uniform_int(seed, stream, n, lo, hi, device="cpu", start=0):
    """Integers uniform over [lo, hi] (inclusive), int64."""
    r = _shr(rand64(seed, stream, n, device, start), 1)
    return lo + torch.remainder(r, hi - lo + 1)


def as_u64(t):
    """Reinterpret an int64 tensor as uint64 (same bits)."""
    return t.view(torch.uint64)


def keys_uniform_over(seed, stream, n, D, device="cpu", start=0):
    """uint64 keys uniform over D distinct values spread by mix64 (int64 bits)."""
    j = uniform_int(seed, stream, n, 0, D - 1, device, start)
    return mix64(j)


# --------------------------------------------------------------------------
# Workload recipes.  Each returns a dict with
#   key_cols: list of unsigned tensors (column 0 most significant)
#   payload:  list of int64 tensors
#   aggs:     list of (op, col) with op 0=COUNT 1=SUM 2=MIN 3=MAX
#   M:        memory budget in rows
# --------------------------------------------------------------------------
COUNT, SUM, MIN, MAX = 0, 1, 2, 3


def config1(n=1 << 20, seed=1, device="cpu", D=10_000, M=65_536):
    k = keys_uniform_over(seed, 1, n, D, device)
    p = uniform_int(seed, 2, n, -1000, 1000, device)
    return dict(name="c1", key_cols=[as_u64(k)], payload=[p],
                aggs=[(COUNT, 0), (SUM, 0), (MIN, 0), (MAX, 0)], M=M, D=D)


C2_COMBOS = ((0, 0), (0, 1), (1, 0), (2, 1))
C2_CUTS = (49, 74, 98)  # cumulative percent: 49 / 25 / 24 / 2


def config2(n=1 << 28, seed=1, device="cpu", M=None):
    u = uniform_int(seed, 3, n, 0, 99, device)
    sel = (u >= C2_CUTS[0]).to(torch.int64) + (u >= C2_CUTS[1]).to(torch.int64) \
        + (u >= C2_CUTS[2]).to(torch.int64)
    c0 = torch.tensor([a for a, _ in C2_COMBOS], dtype=torch.int64, device=device)[sel]
    c1 = torch.tensor([b for _, b in C2_COMBOS], dtype=torch.int64, device=device)[sel]
    pay = [uniform_int(seed, 10 + c, n, 0, 10**7 - 1, device) for c in range(4)]
    aggs = [(COUNT, 0)]
    for c in range(4):
        aggs += [(SUM, c), (MIN, c), (MAX, c)]
    return dict(name="c2", key_cols=[c0.to(torch.uint8), c1.to(torch.uint8)], payload=pay,
                aggs=aggs, M=n if M is None else M)


def config3(n=1 << 29, seed=1, device="cpu", D=1 << 28, M=1 << 25):
    k = keys_uniform_over(seed, 4, n, D, device)
    p = uniform_int(seed, 5, n, -10**9, 10**9, device)
    return dict(name="c3", key_cols=[as_u64(k)], payload=[p], aggs=[(COUNT, 0), (SUM, 0)],
                M=M, D=D)


def log_uniform_int(rng, lo, hi, size=None):
    """exp(U(log lo, log hi)) rounded down, in [lo, hi]."""
    x = np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))
    return np.clip(np.floor(x).astype(np.int64), lo, hi)


def zipf_cdf(D, s=1.1):
    w = np.arange(1, D + 1, dtype=np.float64) ** (-s)
    c = np.cumsum(w)
    return c / c[-1]


def zipf_ranks(seed, stream, n, D, s=1.1, device="cpu"):
    """Ranks in [1, D] with P(r) proportional to r^-s (inverse CDF table)."""
    cdf = torch.tensor(zipf_cdf(D, s), dtype=torch.float64, device=device)
    r = _shr(rand64(seed, stream, n, device), 11).to(torch.float64) * (1.0 / (1 << 53))
    idx = torch.searchsorted(cdf, r, right=True)
    return torch.clamp(idx, max=D - 1) + 1


def config4_instances(count=4096, seed=1, lo=1 << 10, hi=1 << 22, dlo=16, dhi=1 << 20):
    """Per-instance (rows, domain, seed) for the batched workload."""
    rng = np.random.default_rng(seed)
    rows = log_uniform_int(rng, lo, hi, count)
    dom = log_uniform_int(rng, dlo, dhi, count)
    seeds = [int(x) for x in rng.integers(1, 2**62, size=count)]
    return [dict(rows=int(r), D=int(d), seed=s) for r, d, s in zip(rows, dom, seeds)]


def config4_instance(inst, device="cpu"):
    n, D, seed = inst["rows"], inst["D"], inst["seed"]
    ranks = zipf_ranks(seed, 1, n, D, 1.1, device)
    k = fmix32(ranks).to(torch.uint32)
    p = uniform_int(seed, 2, n, -1000, 1000, device)
    return dict(key_cols=[k], payload=[p], aggs=[(COUNT, 0), (SUM, 0), (MIN, 0), (MAX, 0)],
                M=n)


def config5_requests(count=10_000, seed=1, lo=1 << 10, hi=1 << 24, rate=None):
    """Per-request (rows, distinct domain, seed, arrival time) for serving."""
    rng = np.random.default_rng(seed)
    rows = log_uniform_int(rng, lo, hi, count)
    ratio = np.exp(rng.uniform(math.log(0.001), math.log(1.0), size=count))
    dom = np.maximum(1, np.floor(rows * ratio)).astype(np.int64)
    seeds = [int(x) for x in rng.integers(1, 2**62, size=count)]
    gaps = rng.exponential(1.0, size=count)
    arr = np.cumsum(gaps) / (rate if rate else 1.0)
    return [dict(rows=int(r), D=int(d), seed=s, arrival=float(a))
            for r, d, s, a in zip(rows, dom, seeds, arr)]


def config5_pool(device="cpu", seed=1, rows=1 << 24):
    """Device-resident pools from which config5_pooled_request cuts requests
    with two kernels each, for replaying a request stream faster than the
    GPU serves it: T = mix64(0 .. rows-1) (the key values), R = uniform
    draws, P0 / P1 = payloads of the config-5 ranges.  Slots of R beyond
    `rows` wrap, so any request of up to `rows` rows fits."""
    return dict(rows=rows, T=mix64(torch.arange(rows, dtype=torch.int64, device=device)),
                R=_shr(rand64(seed, 7, 2 * rows, device), 1),
                P0=uniform_int(seed, 8, 2 * rows, -1000, 1000, device),
                P1=uniform_int(seed, 9, 2 * rows, 0, 10**7 - 1, device))


def config5_pooled_request(pool, req):
    """A config-5 request from the pools: keys uniform over D = req["D"]
    mix64-spread values (T[R mod D]), payloads as in config5_request; the
    request's seed picks where in the pools its rows start."""
    n, D, seed = req["rows"], req["D"], req["seed"]
    assert n <= pool["rows"] and D <= pool["rows"]
    o = seed % pool["rows"]
    k = pool["T"][torch.remainder(pool["R"][o:o + n], D)]
    p0 = pool["P0"][o:o + n]
    p1 = pool["P1"][(o + 12345) % pool["rows"]:(o + 12345) % pool["rows"] + n]
    aggs = [(COUNT, 0), (SUM, 0), (MIN, 0), (MAX, 0), (SUM, 1), (MIN, 1), (MAX, 1)]
    return dict(key_cols=[as_u64(k)], payload=[p0, p1], aggs=aggs, M=1 << 22)


def config5_request(req, device="cpu", M=1 << 22):
    n, D, seed = req["rows"], req["D"], req["seed"]
    k = keys_uniform_over(seed, 1, n, D, device)
    p0 = uniform_int(seed, 2, n, -1000, 1000, device)
    p1 = uniform_int(seed, 3, n, 0, 10**7 - 1, device)
    aggs = [(COUNT, 0), (SUM, 0), (MIN, 0), (MAX, 0), (SUM, 1), (MIN, 1), (MAX, 1)]
    return dict(key_cols=[as_u64(k)], payload=[p0, p1], aggs=aggs, M=M)


def edge_keys(kind, n, seed=7, device="cpu"):
    """Adversarial key columns (uint64) for edge-case tests."""
    if kind == "all_equal":
        return torch.full((n,), 42, dtype=torch.int64, device=device).view(torch.uint64)
    if kind == "distinct":
        return as_u64(mix64(torch.arange(n, dtype=torch.int64, device=device) + seed))
    if kind == "sorted":
        return torch.arange(n, dtype=torch.int64, device=device).view(torch.uint64)
    if kind == "reverse":
        return torch.arange(n - 1, -1, -1, dtype=torch.int64, device=device).view(torch.uint64)
    if kind == "small_int":
        return uniform_int(seed, 9, n, 0, max(1, n // 3), device).view(torch.uint64)
    if kind == "extremes":
        r = uniform_int(seed, 9, n, 0, 3, device)
        vals = torch.tensor([0, -1, _s64(1 << 63), _s64((1 << 63) - 1)], dtype=torch.int64,
                            device=device)
        return vals[r].view(torch.uint64)
    if kind == "same_digit":
        # every byte but the lowest equal: all keys share 56 high bits
        r = uniform_int(seed, 9, n, 0, 255, device)
        return (r | _s64(0xABABABABABABAB00)).view(torch.uint64)
    if kind == "clustered":
        # dense clusters of consecutive integers at a few far-apart bases
        c = uniform_int(seed, 9, n, 0, 3, device)
        off = uniform_int(seed, 10, n, 0, max(1, n // 2), device)
        return (mix64(c) + off).view(torch.uint64)
    if kind == "heavy_light":
        # 40 heavy keys (30 % of the rows: hundreds of rows each) among light
        # keys of about one row each, interleaved in key order
        u = uniform_int(seed, 9, n, 0, 99, device)
        heavy = uniform_int(seed, 10, n, 0, 39, device)
        light = uniform_int(seed, 11, n, 40, 40 + n, device)
        return as_u64(mix64(torch.where(u < 30, heavy, light)))
    raise ValueError(kind)

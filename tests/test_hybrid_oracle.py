"""Hybrid run generation (Sec. 5.2.3) in the oracle: memory split between an
index that absorbs a resident key range and read-sort-write runs for the
rest, then one wide merge.  Pinned by the plain grouping, the paper's worked
example, the two degenerate splits and a brute-force count of every run."""
import math

import numpy as np
import pytest
import torch

import datagen
import oracle
from oracle import spill_model as sm

AGGS = [(oracle.COUNT, 0), (oracle.SUM, 0), (oracle.MIN, 0), (oracle.MAX, 1)]


def case(n, D, seed):
    k = datagen.keys_uniform_over(seed, 1, n, D).view(torch.uint64).numpy()
    pay = [datagen.uniform_int(seed, 2, n, -1000, 1000).numpy(), datagen.rand64(seed, 3, n).numpy()]
    return k, pay


def same(a, b):
    (ak, aa), (bk, ba) = a, b
    return np.array_equal(ak, bk) and all(np.array_equal(x, y) for x, y in zip(aa, ba))


@pytest.mark.parametrize("M,F,D,n", [(4000, 10, 11_000, 200_003), (500, 4, 1_900, 50_001),
                                     (1000, 10, 900, 30_000), (64, 2, 120, 5_000)])
def test_hybrid_output_is_the_grouping(M, F, D, n):
    k, pay = case(n, D, 5)
    O = len(np.unique(k))
    f = min(F, sm.hybrid_fanout(O, M, 1))
    b = oracle.hybrid_bound(k, M, F, f)
    runs, absorbed, resident, out = oracle.hybrid_runs(k, pay, AGGS, M, F, f, b)
    assert same(out, oracle.groupby(k, pay, AGGS))
    assert resident <= (1 - f / F) * M  # the index never holds more than its share
    assert absorbed == (int((k <= np.uint64(b)).sum()) if b is not None else 0)


def test_hybrid_paper_example():
    """Sec. 5.2.3 with M = 4,000 rows: F = 10, O = 2 3/4 M, I = 100 O, page
    P = 1 row.  f = 2; the index (8/10 of memory) keeps 3,200 keys = 16/55 of
    the output (printed as 3/11); the runs take the other 39/55 of the input
    (printed 8/11: 200 M of 275 M), in runs of 0.2 M input rows -- about
    1,000 runs; O <= F M, so one wide merge step takes them all."""
    M, F, P = 4000, 10, 1
    O = 11 * M // 4
    I = 100 * O
    assert sm.hybrid_fanout(O, M, P) == 2
    k, pay = case(I, O, 11)
    assert len(np.unique(k)) == O  # every key drawn (P(missing) ~ e^-100)
    f = 2
    b = oracle.hybrid_bound(k, M, F, f)
    runs, absorbed, resident, out = oracle.hybrid_runs(k, pay, AGGS, M, F, f, b)
    assert resident == 3200
    spilled = I - absorbed
    frac = 1 - resident / O                       # uniform keys: share of rows outside the index
    assert frac == pytest.approx(39 / 55)
    sd = math.sqrt(I * frac * (1 - frac))
    assert abs(spilled - I * frac) < 5 * sd
    assert len(runs) == math.ceil(spilled / (f / F * M))
    assert abs(len(runs) - 1000) / 1000 < 0.03  # "there will be 1,000 runs"
    assert O <= F * M                              # a single wide merge step suffices
    assert same(out, oracle.groupby(k, pay, AGGS))


def test_hybrid_no_spill_when_output_fits():
    """O <= M: f = 0, the index absorbs everything, no run is written."""
    k, pay = case(40_000, 700, 2)
    M, F = 1000, 10
    f = sm.hybrid_fanout(len(np.unique(k)), M, 1)
    assert f == 0
    b = oracle.hybrid_bound(k, M, F, f)
    runs, absorbed, resident, out = oracle.hybrid_runs(k, pay, AGGS, M, F, f, b)
    assert runs == [] and absorbed == len(k) and resident == 700
    assert same(out, oracle.groupby(k, pay, AGGS))


def test_hybrid_full_partitioning():
    """f = F: no index at all, runs of M input rows (not a true hybrid)."""
    k, pay = case(30_000, 5_000, 4)
    M, F = 700, 8
    b = oracle.hybrid_bound(k, M, F, F)
    assert b is None
    runs, absorbed, resident, out = oracle.hybrid_runs(k, pay, AGGS, M, F, F, b)
    assert absorbed == 0 and resident == 0
    assert len(runs) == math.ceil(len(k) / M)
    assert same(out, oracle.groupby(k, pay, AGGS))


def test_hybrid_runs_brute_force():
    """Every run holds the distinct keys of its batch of spilled rows, in
    input order, batches of f/F * M rows."""
    k, pay = case(9_001, 400, 7)
    M, F, f = 200, 5, 2
    b = oracle.hybrid_bound(k, M, F, f)
    runs, absorbed, resident, _ = oracle.hybrid_runs(k, pay, AGGS, M, F, f, b)
    spilled = [int(x) for x in k if int(x) > b]
    m = int(f / F * M)
    expect = [len(set(spilled[i:i + m])) for i in range(0, len(spilled), m)]
    assert runs == expect
    assert resident == len({int(x) for x in k if int(x) <= b}) == int((1 - f / F) * M)


def test_hybrid_top_key_stays_resident():
    """Every key fits the index, the largest being 2^64 - 1: it stays
    resident with the others, nothing spills, and the resident count is
    the whole output."""
    rng = np.random.default_rng(3)
    k = rng.integers(0, 50, 5_000, dtype=np.uint64)
    k[::97] = np.uint64((1 << 64) - 1)
    pay = [rng.integers(-9, 9, 5_000), rng.integers(-9, 9, 5_000)]
    M, F, f = 1000, 10, 1
    b = oracle.hybrid_bound(k, M, F, f)
    assert b == (1 << 64) - 1
    runs, absorbed, resident, out = oracle.hybrid_runs(k, pay, AGGS, M, F, f, b)
    assert runs == [] and absorbed == len(k) and resident == len(np.unique(k)) == 51
    assert same(out, oracle.groupby(k, pay, AGGS))

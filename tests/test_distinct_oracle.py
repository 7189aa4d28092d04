"""Pins of the oracle's count(distinct u) per group (duplicate removal
followed by grouping, Sec. 7): brute force with Python sets on small
inputs, invariants, and the special cases that reduce to plain grouping."""
import numpy as np
import pytest

import oracle

AGGS = [(0, 0), (1, 0), (2, 0), (3, 0)]


@pytest.mark.parametrize("seed", range(8))
def test_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(0, 400))
    g = rng.integers(0, 12, n).astype(np.uint16)
    u = rng.integers(0, 30, n).astype(np.uint32)
    p = rng.integers(-50, 50, n).astype(np.int64)
    (gk,), dist, aggs = oracle.count_distinct([g], u, [p], AGGS)
    groups = sorted(set(g.tolist()))
    assert gk.tolist() == groups
    for i, x in enumerate(groups):
        sel = g == x
        assert dist[i] == len(set(u[sel].tolist()))
        assert aggs[0][i] == sel.sum() and aggs[1][i] == p[sel].sum()
        assert aggs[2][i] == p[sel].min() and aggs[3][i] == p[sel].max()


def test_invariants_and_special_cases():
    rng = np.random.default_rng(7)
    n = 50_000
    g = rng.integers(0, 300, n).astype(np.uint32)
    u = rng.integers(0, 2_000, n).astype(np.uint32)
    p = rng.integers(-10**9, 10**9, n).astype(np.int64)
    (gk,), dist, aggs = oracle.count_distinct([g], u, [p], AGGS)
    assert (dist <= aggs[0]).all() and (dist >= 1).all()
    pairs = np.unique((g.astype(np.uint64) << np.uint64(32)) | u.astype(np.uint64))
    assert dist.sum() == len(pairs)
    # the other aggregates are those of grouping by g alone
    rk, ra = oracle.groupby(oracle.normalize([g]), [p], AGGS)
    assert (rk == gk).all() and all((a == b).all() for a, b in zip(aggs, ra))
    # u constant: one distinct value per group; u = row id: distinct = count
    (_,), d1, a1 = oracle.count_distinct([g], np.zeros(n, np.uint8), [p], AGGS)
    assert (d1 == 1).all()
    (_,), d2, a2 = oracle.count_distinct([g], np.arange(n, dtype=np.uint32), [p], AGGS)
    assert (d2 == a2[0]).all()

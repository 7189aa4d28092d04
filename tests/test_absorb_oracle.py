"""Pins of the oracle's absorbing-index run generation (Sec. 3, Sec. 6.1):
brute force on tiny inputs (a dict and a Python list, written
independently), the no-spill condition O <= M, the read-sort-write run
sizes, a coupon-collector closed form for the spill of uniform keys, and
bounds against the per-batch run policy."""
import math
import random

import numpy as np
import pytest

import oracle

AGGS = [(0, 0), (1, 0)]


def brute(keys, M, B):
    """Row-by-row statement of the policy: batches of B rows, each batch's
    distinct keys in ascending order, absorbed if present, else inserted
    while fewer than M keys are held, else the held keys become a run."""
    runs, held = [], {}
    for s in range(0, len(keys), B):
        for x in sorted(set(keys[s:s + B])):
            if x in held:
                held[x] += 1
                continue
            if len(held) == M:
                runs.append(len(held))
                held = {}
            held[x] = 1
    if runs:
        runs.append(len(held))
    return runs, len(held)


@pytest.mark.parametrize("seed", range(12))
def test_matches_brute_force(seed):
    rng = random.Random(seed)
    n = rng.randint(0, 300)
    D = rng.randint(1, 120)
    M = rng.randint(1, 40)
    B = rng.randint(1, 50)
    keys = [rng.randrange(D) * 7919 % 1000003 for _ in range(n)]
    pay = np.array([rng.randint(-5, 5) for _ in range(n)], dtype=np.int64)
    got = oracle.absorb_runs(np.array(keys, dtype=np.uint64), [pay], AGGS, M, B)
    assert got == brute(keys, M, B)


@pytest.mark.parametrize("B", [1, 7, 1000, 50_000])
def test_no_spill_when_output_fits(B):
    rng = np.random.default_rng(3)
    O, M = 900, 1000
    keys = rng.integers(0, O, 50_000).astype(np.uint64)
    runs, left = oracle.absorb_runs(keys, [keys.astype(np.int64)], AGGS, M, B)
    assert runs == [] and left == len(np.unique(keys))


def test_runs_hold_memory_size():
    rng = np.random.default_rng(5)
    keys = rng.integers(0, 5000, 40_000).astype(np.uint64)
    runs, left = oracle.absorb_runs(keys, [keys.astype(np.int64)], AGGS, 700, 333)
    assert len(runs) > 2 and all(r == 700 for r in runs[:-1]) and runs[-1] == left
    # never more spill than one run per batch of its distinct keys
    per_batch = sum(len(np.unique(keys[s:s + 333])) for s in range(0, len(keys), 333))
    assert sum(runs) <= per_batch
    assert sum(runs) >= len(np.unique(keys))


@pytest.mark.parametrize("O,M", [(2000, 1000), (3000, 1000), (4000, 3000)])
def test_uniform_spill_closed_form(O, M):
    # row at a time (B = 1), keys uniform over O values: a run closes when
    # the (M+1)-th distinct key since the last run appears, so rows per run
    # = the coupon-collector time for M of O coupons, O (H_O - H_{O-M})
    n = 400_000
    rng = np.random.default_rng(O + M)
    keys = rng.integers(0, O, n).astype(np.uint64)
    runs, _ = oracle.absorb_runs(keys, [keys.astype(np.int64)], AGGS, M, 1)
    H = lambda k: sum(1.0 / i for i in range(1, k + 1))
    per_run = O * (H(O) - H(O - M))
    assert len(runs) == pytest.approx(n / per_run, rel=0.03)

"""Hybrid run generation on the GPU (SGAGG_OPT_POLICY 2, Sec. 5.2.3) against
the oracle's statement of it: memory fraction 1 - f/F an in-memory index of
the lowest keys (their rows absorbed, never spilled), fraction f/F read-sort-
write runs of f/F * M rows over the other rows, one wide merge.  The grouped
output bit for bit, the rows the index absorbed and its keys, and every
run's row count, in order; f = 0 (everything resident) and f = F (no index)
included, and a resident range ending at the largest key, 2^64 - 1."""
import numpy as np
import pytest
import torch

import datagen
import oracle
from oracle import spill_model as sm
from paper_2010_00152_gb300 import sgagg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
AGGS = [(oracle.COUNT, 0), (oracle.SUM, 0), (oracle.MIN, 0), (oracle.MAX, 1)]


def case(n, D, seed):
    k = datagen.keys_uniform_over(seed, 1, n, D).view(torch.uint64)
    pay = [datagen.uniform_int(seed, 2, n, -1000, 1000), datagen.rand64(seed, 3, n)]
    return k, pay


def run(k, pay, M, F, f, last=None, **extra):
    opts = dict(policy=2, hybrid_fanin=F, hybrid_f=f, **extra)
    if last is not None:
        opts["hybrid_last"] = last
    agg = sgagg.Aggregator(M, **opts)
    try:
        ok, oa = agg.aggregate([k.to(DEV)], [p.to(DEV) for p in pay], AGGS)
        return ok[0].cpu().numpy(), [a.cpu().numpy() for a in oa], agg.stats(), agg.run_sizes()
    finally:
        agg.close()


def check(k, pay, M, F, f, last, **extra):
    gk, ga, st, sizes = run(k, pay, M, F, f, last, **extra)
    kn, pn = k.numpy(), [p.numpy() for p in pay]
    runs, absorbed, resident, (rk, ra) = oracle.hybrid_runs(kn, pn, AGGS, M, F, f, last)
    np.testing.assert_array_equal(gk, rk)
    for a, b in zip(ga, ra):
        np.testing.assert_array_equal(a, b)
    assert st["resident_rows"] == absorbed and st["resident_keys"] == resident
    assert st["hybrid_f"] == f
    assert sizes[:len(runs)] == runs and st["runs"] >= len(runs)
    return st, runs


@pytest.mark.parametrize("M,F,D,n", [(4000, 10, 11_000, 200_003), (500, 4, 1_900, 50_001),
                                     (1000, 10, 900, 30_000), (64, 2, 120, 5_000)])
def test_hybrid_matches_oracle(M, F, D, n):
    k, pay = case(n, D, 5)
    O = len(np.unique(k.numpy()))
    f = min(F, sm.hybrid_fanout(O, M, 1))
    last = oracle.hybrid_bound(k.numpy(), M, F, f)
    st, runs = check(k, pay, M, F, f, last)
    assert st["runs"] == len(runs)  # at most 256 runs: one wide merge takes them all


@pytest.mark.parametrize("one_pass", [1, 0])
def test_hybrid_runs_in_one_pass(one_pass):
    """Spilled rows in runs of more than one chunk (f/F * M = 50,000 rows):
    their runs generated in one pass, or a batch at a time.  The output and
    every run's row count equal the oracle's."""
    n, D, M, F, f = 400_003, 150_000, 100_000, 4, 2
    k, pay = case(n, D, 7)
    last = oracle.hybrid_bound(k.numpy(), M, F, f)
    st, runs = check(k, pay, M, F, f, last, one_pass=one_pass)
    assert len(runs) > 1 and st["one_pass"] == one_pass


def test_hybrid_paper_example_shape():
    """Sec. 5.2.3's example at M = 4,000: F = 10, O = 2 3/4 M, I = 100 O,
    f = 2: the index keeps 3,200 keys, about 1,000 runs of 0.2 M rows, one
    wide merge (more runs than one merge takes first get preliminary merges:
    the oracle's runs are the first ones written)."""
    M, F, f = 4000, 10, 2
    O = 11 * M // 4
    k, pay = case(100 * O, O, 11)
    last = oracle.hybrid_bound(k.numpy(), M, F, f)
    st, runs = check(k, pay, M, F, f, last)
    assert st["resident_keys"] == 3200 and abs(len(runs) - 1000) / 1000 < 0.03


@pytest.mark.parametrize("which", ["f0", "fF"])
def test_hybrid_degenerate_splits(which):
    k, pay = case(40_000, 700 if which == "f0" else 5_000, 2)
    M, F = 1000, 8
    f = 0 if which == "f0" else F
    last = oracle.hybrid_bound(k.numpy(), M, F, f)
    st, runs = check(k, pay, M, F, f, last)
    if which == "f0":
        assert runs == [] and st["runs"] == 0 and st["resident_rows"] == 40_000
    else:
        assert last is None and st["resident_rows"] == 0 and len(runs) == 40


def test_hybrid_top_key_resident():
    rng = np.random.default_rng(3)
    kn = rng.integers(0, 50, 20_000, dtype=np.uint64)
    kn[::97] = np.uint64((1 << 64) - 1)
    k = torch.from_numpy(kn.view(np.int64)).view(torch.uint64)
    pay = [torch.from_numpy(rng.integers(-9, 9, 20_000)), torch.from_numpy(rng.integers(-9, 9, 20_000))]
    M, F, f = 1000, 10, 1
    last = oracle.hybrid_bound(kn, M, F, f)
    assert last == (1 << 64) - 1
    st, runs = check(k, pay, M, F, f, last)
    assert runs == [] and st["resident_keys"] == 51


def test_hybrid_estimated_resident_range():
    """Without a given range the GPU estimates it on its key sample; the
    output is exact, the index holds the lowest keys, and the runs are those
    the oracle writes for the same resident range."""
    M, F = 3000, 10
    k, pay = case(300_000, 9000, 8)
    gk, ga, st, sizes = run(k, pay, M, F, -1)
    kn = k.numpy()
    uk = np.unique(kn)
    f = st["hybrid_f"]
    assert 0 < f <= F
    rk_ = st["resident_keys"]
    last = int(uk[rk_ - 1]) if rk_ > 0 else None
    runs, absorbed, resident, (rk, ra) = oracle.hybrid_runs(kn, [p.numpy() for p in pay], AGGS, M, F, f, last)
    np.testing.assert_array_equal(gk, rk)
    for a, b in zip(ga, ra):
        np.testing.assert_array_equal(a, b)
    assert st["resident_rows"] == absorbed and sizes[:len(runs)] == runs
    assert abs(rk_ - (1 - f / F) * M) < 0.15 * M  # the sample's estimate of the index's share

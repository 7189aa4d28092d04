"""Absorbing-index run generation on the GPU (SGAGG_OPT_POLICY = 1) against
the oracle: the grouped result bit for bit, and the runs themselves (how
many, rows in each) exactly as the oracle's statement of the policy writes
them; no run at all when the output fits the budget."""
import numpy as np
import pytest
import torch

import datagen
import oracle
from paper_2010_00152_gb300 import sgagg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
AGG4 = [(0, 0), (1, 0), (2, 0), (3, 0)]


def run_gpu(c, M, Bz, **opts):
    agg = sgagg.Aggregator(M, policy=1, absorb_batch=Bz, **opts)
    try:
        ok, oa = agg.aggregate(c["key_cols"], c["payload"], c["aggs"])
        return [k.cpu().numpy() for k in ok], [a.cpu().numpy() for a in oa], agg.stats()
    finally:
        agg.close()


def check(c, M, Bz, **opts):
    gk, ga, st = run_gpu(c, M, Bz, **opts)
    kc = [k.cpu().numpy() for k in c["key_cols"]]
    pc = [p.cpu().numpy() for p in c["payload"]]
    rk, ra = oracle.aggregate(kc, pc, c["aggs"])
    np.testing.assert_array_equal(gk[0], rk[0])
    for a, r in zip(ga, ra):
        np.testing.assert_array_equal(a, r)
    runs, left = oracle.absorb_runs(oracle.normalize(kc), pc, c["aggs"], M, Bz)
    return st, runs, left


@pytest.mark.parametrize("n,D,M,Bz", [
    (200_000, 50_000, 16_384, 4_096),     # the index overflows in most batches
    (200_000, 50_000, 16_384, 20_000),    # batches bigger than a chunk
    (150_001, 150_001, 30_000, 30_000),   # nearly all keys distinct
    (120_000, 9_000, 10_000, 3_000),      # output just fits: absorbed
    (100_000, 40_000, 5_000, 100_000),    # one batch, many full indexes
    (7_000, 2_000, 1, 7),                 # budget of one key
])
def test_absorbing_matches_oracle(n, D, M, Bz):
    c = datagen.config1(n=n, D=D, M=M, device=DEV)
    c["aggs"] = AGG4
    st, runs, left = check(c, M, Bz)
    assert st["batches"] == (n + Bz - 1) // Bz
    if len(runs) <= 256:
        assert st["runs"] == len(runs)
        assert st["run_rows"] == sum(runs)
    else:  # more runs than one merge takes: the preliminary merges add their own runs
        assert st["runs"] > len(runs) and st["run_rows"] > sum(runs)


def test_no_runs_when_output_fits():
    c = datagen.config1(n=1 << 20, D=10_000, M=65_536, device=DEV)
    st, runs, left = check(c, 65_536, 65_536)
    assert runs == [] and st["runs"] == 0 and st["run_rows"] == 0 and st["out_rows"] == left == 10_000


def test_absorbing_with_preliminary_merges():
    c = datagen.config1(n=300_000, D=120_000, M=8_192, device=DEV)
    c["aggs"] = AGG4
    st, runs, left = check(c, 8_192, 8_192, fanin_cap=3)
    assert len(runs) > 3


def test_absorbing_composite_keys_and_wide_payloads():
    c = datagen.config2(n=300_000, device=DEV)
    check(c, 2, 50_000)  # 4 distinct keys against a 2-key index
    k = datagen.keys_uniform_over(9, 1, 90_000, 30_000, DEV)
    c = dict(key_cols=[datagen.as_u64(k)], payload=[datagen.uniform_int(9, 2, 90_000, -10**12, 10**12, DEV),
                                                      datagen.uniform_int(9, 3, 90_000, 0, 5, DEV)],
             aggs=[(1, 0), (0, 0), (3, 1), (2, 0), (1, 1)])
    check(c, 7_000, 9_000)

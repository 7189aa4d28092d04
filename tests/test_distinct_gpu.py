"""count(distinct u) per group on the GPU (one grouping on (g, u), one
in-stream regroup on g) against the oracle, bit for bit."""
import numpy as np
import pytest
import torch

import datagen
import oracle
from paper_2010_00152_gb300 import sgagg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
AGGS = [(0, 0), (1, 0), (2, 1), (3, 1)]


def case(n, G, U, gdtype, udtype, seed):
    g = datagen.uniform_int(seed, 1, n, 0, G - 1, DEV)
    u = datagen.uniform_int(seed, 2, n, 0, U - 1, DEV)
    p0 = datagen.uniform_int(seed, 3, n, -10**9, 10**9, DEV)
    p1 = datagen.uniform_int(seed, 4, n, -1000, 1000, DEV)
    return g.to(gdtype), u.to(udtype), [p0, p1]


@pytest.mark.parametrize("n,G,U,gd,ud,M", [
    (300_000, 1_000, 5_000, torch.uint16, torch.uint32, 1 << 20),   # one batch
    (400_000, 70_000, 50, torch.uint32, torch.uint8, 60_000),       # runs + wide merge
    (200_001, 3, 200_000, torch.uint8, torch.uint32, 30_000),       # few huge groups
    (9_000, 9_000, 2, torch.uint16, torch.uint16, 1 << 20),         # one chunk
    (0, 1, 1, torch.uint16, torch.uint32, 1024),                    # empty
])
def test_count_distinct_matches_oracle(n, G, U, gd, ud, M):
    g, u, pay = case(n, G, U, gd, ud, 5)
    agg = sgagg.Aggregator(M)
    try:
        ok, od, oa = agg.aggregate_distinct([g], u, pay, AGGS)
    finally:
        agg.close()
    (rk,), rd, ra = oracle.count_distinct([g.cpu().numpy()], u.cpu().numpy(), [p.cpu().numpy() for p in pay], AGGS)
    np.testing.assert_array_equal(ok[0].cpu().numpy(), rk)
    np.testing.assert_array_equal(od.cpu().numpy(), rd)
    for a, r in zip(oa, ra):
        np.testing.assert_array_equal(a.cpu().numpy(), r)


def test_count_distinct_composite_group_and_capacity():
    n = 250_000
    c = datagen.config2(n=n, device=DEV)
    u = datagen.uniform_int(3, 9, n, 0, 40_000, DEV).to(torch.uint32)
    pay = c["payload"][:2]
    agg = sgagg.Aggregator(50_000)
    try:
        ok, od, oa = agg.aggregate_distinct(c["key_cols"], u, pay, AGGS)
        with pytest.raises(sgagg.SgaggError) as e:
            agg.aggregate_distinct(c["key_cols"], u, pay, AGGS, capacity=2)
        assert e.value.status == sgagg.SGAGG_ECAPACITY
    finally:
        agg.close()
    rks, rd, ra = oracle.count_distinct([k.cpu().numpy() for k in c["key_cols"]], u.cpu().numpy(),
                                        [p.cpu().numpy() for p in pay], AGGS)
    for a, b in zip(ok, rks):
        np.testing.assert_array_equal(a.cpu().numpy(), b)
    np.testing.assert_array_equal(od.cpu().numpy(), rd)
    for a, r in zip(oa, ra):
        np.testing.assert_array_equal(a.cpu().numpy(), r)

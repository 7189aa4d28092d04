"""The 512M-row workload at its full size, in the configuration the benchmark
times: 2^29 rows, uint64 keys uniform over 2^28 values, one payload, count
and sum, a memory budget of 2^25 rows (16 runs and one wide merge).

The oracle cannot group 2^29 rows in seconds, so the output is checked by
properties that hold at any size -- keys strictly ascending, counts summing
to the input rows, sums summing to the payload sum (|sum| < 2^63 here, so
nothing wraps), every sampled input key present -- and by the oracle on
1,000 sampled output groups, each recomputed from all of its input rows.
Collected late: a run stopping at the first failure has run the smaller
cases first.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle
from paper_2010_00152_gb300 import sgagg

pytestmark = pytest.mark.gpu
SIGN = -(1 << 63)


def ordered(k64):
    """int64 keys whose signed order is the unsigned order of the keys."""
    return k64 ^ SIGN


def test_c3_full_size_sampled():
    c = datagen.config3(device="cuda")
    kin = c["key_cols"][0].view(torch.int64)
    pay = c["payload"][0]
    n = kin.numel()
    agg = sgagg.Aggregator(c["M"])
    try:
        ok, oa = agg.aggregate(c["key_cols"], c["payload"], c["aggs"], capacity=n)
        st = agg.stats()
    finally:
        agg.close()
    kout = ok[0].view(torch.int64)
    rows = kout.numel()
    assert st["runs"] == 16 and st["out_rows"] == rows
    out = ordered(kout)
    assert bool((out[1:] > out[:-1]).all())
    cnt, sm = oa
    assert int(cnt.sum()) == n and int(cnt.min()) >= 1
    assert int(sm.sum()) == int(pay.sum())

    rng = np.random.default_rng(29)
    # every sampled input key is an output key
    ri = torch.from_numpy(rng.integers(0, n, 1000)).to(kin.device)
    probe = ordered(kin[ri])
    pos = torch.searchsorted(out, probe).clamp(max=rows - 1)
    assert bool((out[pos] == probe).all())

    # 1,000 output groups, recomputed by the oracle from all of their rows
    gi = np.unique(rng.integers(0, rows, 3000))[:1000]
    assert len(gi) == 1000
    gi = torch.from_numpy(gi).to(kin.device)
    skeys = out[gi]
    allk = ordered(kin)
    hit = skeys[torch.searchsorted(skeys, allk).clamp(max=999)] == allk
    del allk
    mk = kin[hit].cpu().numpy().view(np.uint64)
    mp = pay[hit].cpu().numpy()
    rk, ra = oracle.groupby(mk, [mp], c["aggs"])
    np.testing.assert_array_equal(rk, kout[gi].cpu().numpy().view(np.uint64))
    for a in range(len(c["aggs"])):
        np.testing.assert_array_equal(ra[a], oa[a][gi].cpu().numpy(), err_msg="aggregate %d" % a)
    del c, kin, pay, ok, oa, kout, out, cnt, sm, hit
    torch.cuda.empty_cache()

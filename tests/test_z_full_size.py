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


def test_c2_full_size_closed_form():
    """The 256M-row report shape at full size (one batch, four key
    combinations): the four output rows equal the direct per-combination
    accumulation (count, and sum / min / max of each payload column over the
    rows of that combination, computed by plain torch reductions), with the
    streaming fold of few keys and with the general sort+fold path; and the
    oracle agrees with the GPU path on the first 2^24 rows."""
    c = datagen.config2(device="cuda")
    n = c["key_cols"][0].numel()
    k0, k1 = c["key_cols"]
    combos = sorted(datagen.C2_COMBOS)
    want = []
    for a, b in combos:
        m = (k0 == a) & (k1 == b)
        row = [int(m.sum())]
        for p in c["payload"]:
            v = p[m]
            row += [int(v.sum()), int(v.min()), int(v.max())]
        want.append(row)
        del m
    want = np.array(want, dtype=np.int64).T  # [aggregate][combination]
    for lowcard in (-1, 0):
        agg = sgagg.Aggregator(c["M"], lowcard=lowcard)
        try:
            ok, oa = agg.aggregate(c["key_cols"], c["payload"], c["aggs"], capacity=16)
            st = agg.stats()
        finally:
            agg.close()
        assert st["out_rows"] == 4 and st["runs"] == 0
        if lowcard == -1:
            assert st["kernels"]["stream"]["launches"] == 2
        got_k = list(zip(ok[0].cpu().tolist(), ok[1].cpu().tolist()))
        assert got_k == combos
        for a in range(len(c["aggs"])):
            np.testing.assert_array_equal(oa[a].cpu().numpy(), want[a], err_msg="lowcard %d agg %d" % (lowcard, a))
    m = 1 << 24
    kc = [k[:m] for k in c["key_cols"]]
    pc = [p[:m] for p in c["payload"]]
    agg = sgagg.Aggregator(m)
    try:
        ok, oa = agg.aggregate(kc, pc, c["aggs"], capacity=16)
    finally:
        agg.close()
    rk, ra = oracle.aggregate([k.cpu().numpy() for k in kc], [p.cpu().numpy() for p in pc], c["aggs"])
    for j in range(2):
        np.testing.assert_array_equal(ok[j].cpu().numpy(), rk[j])
    for a in range(len(c["aggs"])):
        np.testing.assert_array_equal(oa[a].cpu().numpy(), ra[a])
    del c, k0, k1, kc, pc
    torch.cuda.empty_cache()


def test_c4_full_size_batched():
    """The batched workload at full size: 4,096 instances (1K-4M rows each,
    Zipf keys) in one batched call.  Every instance: keys strictly ascending,
    counts summing to its rows, sums summing to its payload sum, min <= max;
    64 instances (the 8 largest and 56 drawn at random) element by element
    against the oracle."""
    specs = datagen.config4_instances(count=4096, seed=1)
    insts = [datagen.config4_instance(sp, device="cuda") for sp in specs]
    aggs = insts[0]["aggs"]
    caps = [max(1, min(sp["rows"], sp["D"])) for sp in specs]
    agg = sgagg.Aggregator(1 << 22)
    try:
        res = agg.aggregate_batched([(c["key_cols"][0], [c["payload"][0]]) for c in insts], aggs,
                                    capacities=caps)
        st = agg.stats()
    finally:
        agg.close()
    assert st["n_rows"] == sum(sp["rows"] for sp in specs)
    for i, (c, r) in enumerate(zip(insts, res)):
        assert r is not None, i
        k = r[0].view(torch.int32).to(torch.int64) & 0xFFFFFFFF  # uint32 keys, in order
        assert bool((k[1:] > k[:-1]).all()), i
        cnt, sm, mn, mx = r[1]
        assert int(cnt.sum()) == specs[i]["rows"], i
        assert int(sm.sum()) == int(c["payload"][0].sum()), i
        assert bool((mn <= mx).all()) and int(cnt.min()) >= 1, i
    rng = np.random.default_rng(44)
    big = sorted(range(len(specs)), key=lambda i: -specs[i]["rows"])[:8]
    rest = [i for i in rng.permutation(len(specs)) if i not in big][:56]
    for i in big + rest:
        c = insts[i]
        rk, ra = oracle.aggregate([c["key_cols"][0].cpu().numpy()], [c["payload"][0].cpu().numpy()], aggs)
        np.testing.assert_array_equal(res[i][0].cpu().numpy(), rk[0], err_msg="instance %d" % i)
        for a in range(len(aggs)):
            np.testing.assert_array_equal(res[i][1][a].cpu().numpy(), ra[a], err_msg="instance %d agg %d" % (i, a))
    del insts, res
    torch.cuda.empty_cache()

"""Failure handling on the GPU without faulting it: a device-side wait that
runs out (a chunk that never publishes, with a short spin limit) becomes
SGAGG_ETIMEOUT and the handle keeps working; an injected allocation failure
becomes SGAGG_ENOMEM at every allocation point, leaks nothing, and the next
call on the same handle is exact."""
import numpy as np
import pytest
import torch

import datagen
import oracle
from paper_2010_00152_gb300 import sgagg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def case(n=200_000, D=50_000, M=1 << 20):
    c = datagen.config1(n=n, D=D, M=M, device=DEV)
    ref = oracle.aggregate([k.cpu().numpy() for k in c["key_cols"]], [p.cpu().numpy() for p in c["payload"]],
                           c["aggs"])
    return c, ref


def same(res, ref):
    ok, oa = res
    np.testing.assert_array_equal(ok[0].cpu().numpy(), ref[0][0])
    for a, r in zip(oa, ref[1]):
        np.testing.assert_array_equal(a.cpu().numpy(), r)


def test_device_wait_times_out_and_handle_recovers():
    c, ref = case()
    agg = sgagg.Aggregator(1 << 20, spin_limit=1 << 12, test_stall=1)
    try:
        with pytest.raises(sgagg.SgaggError) as e:
            agg.aggregate(c["key_cols"], c["payload"], c["aggs"])
        assert e.value.status == sgagg.SGAGG_ETIMEOUT
        same(agg.aggregate(c["key_cols"], c["payload"], c["aggs"]), ref)
    finally:
        agg.close()
    torch.cuda.synchronize()  # the context is still usable


def test_merge_wait_times_out_and_handle_recovers():
    """The stall hits the wide merge (32 runs, some 2,000 merge tiles): the
    first block of the scan of the tiles' row counts never publishes, the
    other blocks' bounded look-back waits run out; no merge tile writes."""
    c, ref = case(n=4_000_000, D=2_000_000, M=1 << 17)
    agg = sgagg.Aggregator(1 << 17, spin_limit=1 << 12, test_stall=2)
    try:
        with pytest.raises(sgagg.SgaggError) as e:
            agg.aggregate(c["key_cols"], c["payload"], c["aggs"])
        assert e.value.status == sgagg.SGAGG_ETIMEOUT
        st = agg.stats()
        assert st["runs"] > 1 and st["merge_tiles"] > 1024  # run generation finished; the merge timed out
        same(agg.aggregate(c["key_cols"], c["payload"], c["aggs"]), ref)
    finally:
        agg.close()
    torch.cuda.synchronize()


def test_batched_wait_times_out_and_handle_recovers():
    """The stall hits the first sort+fold launch inside a batched call."""
    insts, refs = [], []
    for i, (n, D) in enumerate([(50_000, 3000), (120_000, 40_000), (9_000, 50)]):
        c = datagen.config4_instance(dict(rows=n, D=D, seed=70 + i))
        insts.append((c["key_cols"][0], [c["payload"][0]]))
        refs.append(oracle.aggregate([c["key_cols"][0].numpy()], [c["payload"][0].numpy()], c["aggs"]))
    aggs = datagen.config4_instance(dict(rows=10, D=2, seed=1))["aggs"]
    dev = [(k.to(DEV), [p.to(DEV) for p in pay]) for k, pay in insts]
    agg = sgagg.Aggregator(1 << 20, spin_limit=1 << 12, test_stall=1)
    try:
        with pytest.raises(sgagg.SgaggError) as e:
            agg.aggregate_batched(dev, aggs)
        assert e.value.status == sgagg.SGAGG_ETIMEOUT
        res = agg.aggregate_batched(dev, aggs)
        for r, (rk, ra) in zip(res, refs):
            np.testing.assert_array_equal(r[0].cpu().numpy(), rk[0])
            for a in range(len(ra)):
                np.testing.assert_array_equal(r[1][a].cpu().numpy(), ra[a])
    finally:
        agg.close()
    torch.cuda.synchronize()


@pytest.mark.parametrize("budget", [1 << 20, 1 << 14])
def test_injected_allocation_failure(budget):
    c, ref = case(M=budget)
    warm = sgagg.Aggregator(budget)  # module loading is not a leak
    try:
        same(warm.aggregate(c["key_cols"], c["payload"], c["aggs"]), ref)
    finally:
        warm.close()
    failed = 0
    for k in range(1, 40):
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        free0 = torch.cuda.mem_get_info()[0]
        agg = sgagg.Aggregator(budget, fault_alloc=k)
        try:
            try:
                agg.aggregate(c["key_cols"], c["payload"], c["aggs"])
                hit = False
            except sgagg.SgaggError as e:
                assert e.status == sgagg.SGAGG_ENOMEM
                hit = True
            agg.set_option(sgagg.SGAGG_OPT_FAULT_ALLOC, 0)
            same(agg.aggregate(c["key_cols"], c["payload"], c["aggs"]), ref)
        finally:
            agg.close()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        assert torch.cuda.mem_get_info()[0] >= free0 - (8 << 20)  # nothing leaked
        if not hit:
            break  # every allocation point has been failed once
        failed += 1
    assert failed >= 3

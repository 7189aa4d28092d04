"""The allocation-free entry point (sgagg_aggregate_noalloc).

Some callers cannot allocate device memory at all -- code running inside a
memory-pool or allocator callback, or a process whose device memory a
framework reserved up front.  For them the library has one handle-free entry
point whose scratch is a fixed array in the library's own device memory.  This
file checks it against the ordinary entry point on two calls in a row (the
scratch is reused and must be cleared by each call), and that oversized
inputs are refused.  It is collected last so that a run stopping at the first
failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest
import torch

import datagen
from paper_2010_00152_gb300 import sgagg

pytestmark = pytest.mark.gpu


def _noalloc(keys, pay, aggs, n):
    dev = keys.device
    ok = torch.empty(max(1, n), dtype=keys.dtype, device=dev)
    oa = [torch.empty(max(1, n), dtype=torch.int64, device=dev) for _ in aggs]
    rows = torch.full((1,), -7, dtype=torch.int64, device=dev)
    s = torch.cuda.current_stream(dev).cuda_stream
    sgagg.sgagg_aggregate_noalloc([keys.data_ptr()], [keys.element_size()], [p.data_ptr() for p in pay], n,
                                  aggs, [ok.data_ptr()], [a.data_ptr() for a in oa], n, rows.data_ptr(), s)
    torch.cuda.synchronize()
    r = int(rows.item())
    return ok[:r].cpu().numpy(), [a[:r].cpu().numpy() for a in oa]


def test_noalloc_matches_aggregate_on_two_calls():
    aggs = [(0, 0), (1, 0), (2, 1), (3, 1), (1, 1)]
    for call, (n, D, seed) in enumerate(((8192, 1500, 3), (5003, 40, 4))):
        c = datagen.config1(n=n, seed=seed, D=D)
        keys = c["key_cols"][0].cuda()
        pay = [c["payload"][0].cuda(), datagen.uniform_int(seed, 9, n, -10**12, 10**12).cuda()]
        agg = sgagg.Aggregator(1 << 20)
        try:
            rk, ra = agg.aggregate([keys], pay, aggs)
            rk = rk[0].cpu().numpy()
            ra = [a.cpu().numpy() for a in ra]
        finally:
            agg.close()
        gk, ga = _noalloc(keys, pay, aggs, n)
        np.testing.assert_array_equal(gk, rk, err_msg="call %d keys" % call)
        for a in range(len(aggs)):
            np.testing.assert_array_equal(ga[a], ra[a], err_msg="call %d aggregate %d" % (call, a))


def test_noalloc_refuses_more_rows_than_its_scratch_covers():
    n = sgagg.NOALLOC_MAX_ROWS + 1
    keys = torch.zeros(n, dtype=torch.int64, device="cuda").view(torch.uint64)
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    rows = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(sgagg.SgaggError) as e:
        sgagg.sgagg_aggregate_noalloc([keys.data_ptr()], [8], [], n, [(0, 0)], [out.data_ptr()],
                                      [out.data_ptr()], n, rows.data_ptr(), 0)
    assert e.value.status == sgagg.SGAGG_EINVAL
    assert "8192" in str(e.value)

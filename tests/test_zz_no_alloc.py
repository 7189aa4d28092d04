"""The allocation-free entry point (sgagg_aggregate_noalloc).

Some callers cannot allocate device memory at all -- code running inside a
memory-pool or allocator callback, or a process whose device memory a
framework reserved up front.  For them the library has one handle-free entry
point whose only scratch is a fixed array in the library's own device memory.
This file checks it through the C ABI against the CPU oracle on two calls in a
row (the scratch is reused and must be cleared by each call), on a composite
key, without aggregates, on an empty input and when the output capacity is
too small (row count -1, nothing written past the capacity); that a warmed-up
call leaves the free device memory unchanged; and that oversized inputs are
refused.  It is collected last so that a run stopping at the first failure
has run every other test first.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle
from paper_2010_00152_gb300 import sgagg

pytestmark = pytest.mark.gpu
SENTINEL = -0x5A5A5A5A5A5A5A5B


def _noalloc(key_cols, pay, aggs, n, capacity=None, pad=4):
    """Run the entry point; outputs are preset to a sentinel with `pad` rows
    past the capacity.  Returns (rows, key outputs, aggregate outputs)."""
    dev = key_cols[0].device if key_cols else torch.device("cuda")
    cap = n if capacity is None else capacity
    ok = [torch.full(((cap + pad) * k.element_size(),), 0x5A, dtype=torch.uint8, device=dev).view(k.dtype)
          for k in key_cols]
    oa = [torch.full((cap + pad,), SENTINEL, dtype=torch.int64, device=dev) for _ in aggs]
    rows = torch.full((1,), -7, dtype=torch.int64, device=dev)
    s = torch.cuda.current_stream(dev).cuda_stream
    sgagg.sgagg_aggregate_noalloc([k.data_ptr() for k in key_cols], [k.element_size() for k in key_cols],
                                  [p.data_ptr() for p in pay], n, aggs, [o.data_ptr() for o in ok],
                                  [a.data_ptr() for a in oa], cap, rows.data_ptr(), s)
    torch.cuda.synchronize()
    return int(rows.item()), [o.cpu().numpy() for o in ok], [a.cpu().numpy() for a in oa]


def _check_against_oracle(key_cols, pay, aggs, n, what):
    rows, gk, ga = _noalloc(key_cols, pay, aggs, n)
    rk, ra = oracle.aggregate([k.cpu().numpy() for k in key_cols], [p.cpu().numpy() for p in pay], aggs)
    assert rows == len(rk[0]), (what, rows, len(rk[0]))
    for c in range(len(rk)):
        np.testing.assert_array_equal(gk[c][:rows], rk[c], err_msg="%s: key column %d" % (what, c))
    for a in range(len(aggs)):
        np.testing.assert_array_equal(ga[a][:rows], ra[a], err_msg="%s: aggregate %d" % (what, a))


def test_noalloc_matches_oracle_on_two_calls():
    aggs = [(0, 0), (1, 0), (2, 1), (3, 1), (1, 1)]
    for call, (n, D, seed) in enumerate(((8192, 1500, 3), (5003, 40, 4))):
        c = datagen.config1(n=n, seed=seed, D=D)
        keys = c["key_cols"][0].cuda()
        pay = [c["payload"][0].cuda(), datagen.uniform_int(seed, 9, n, -10**12, 10**12).cuda()]
        _check_against_oracle([keys], pay, aggs, n, "call %d" % call)


def test_noalloc_composite_key_and_keys_only():
    c = datagen.config2(n=6000, seed=9)
    kc = [k.cuda() for k in c["key_cols"]]
    pc = [p.cuda() for p in c["payload"]]
    _check_against_oracle(kc, pc, c["aggs"], 6000, "composite key")
    _check_against_oracle(kc, pc, [], 6000, "keys only")


def test_noalloc_empty_input():
    keys = torch.empty(0, dtype=torch.int64, device="cuda").view(torch.uint64)
    pay = [torch.empty(0, dtype=torch.int64, device="cuda")]
    rows, gk, ga = _noalloc([keys], pay, [(0, 0), (1, 0)], 0)
    assert rows == 0
    assert (ga[0] == SENTINEL).all() and (ga[1] == SENTINEL).all()


def test_noalloc_capacity_too_small():
    """More distinct keys than out_capacity: the row count is -1 and no row
    at or past the capacity is written."""
    c = datagen.config1(n=4000, seed=5, D=3000)
    keys = c["key_cols"][0].cuda()
    pay = [c["payload"][0].cuda()]
    rows, gk, ga = _noalloc([keys], pay, [(0, 0), (1, 0)], 4000, capacity=100, pad=64)
    assert rows == -1
    assert (gk[0][100:].view(np.uint8) == 0x5A).all()
    for a in ga:
        assert (a[100:] == SENTINEL).all()


def test_noalloc_allocates_nothing():
    """After the first call on the device (its one-time set-up), calls leave
    the device's free memory unchanged: the outputs are allocated before
    the free memory is read, and only the entry point runs in between."""
    n = 8000
    c = datagen.config1(n=n, seed=6, D=700)
    keys = c["key_cols"][0].cuda()
    pay = [c["payload"][0].cuda()]
    aggs = [(0, 0), (1, 0), (2, 0), (3, 0)]
    ok = torch.empty(n, dtype=torch.int64, device="cuda").view(torch.uint64)
    oa = [torch.empty(n, dtype=torch.int64, device="cuda") for _ in aggs]
    rows = torch.empty(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream

    def call():
        sgagg.sgagg_aggregate_noalloc([keys.data_ptr()], [8], [pay[0].data_ptr()], n, aggs, [ok.data_ptr()],
                                      [a.data_ptr() for a in oa], n, rows.data_ptr(), s)

    call()  # the first call on the device does its set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    rk, ra = oracle.aggregate([c["key_cols"][0].numpy()], [c["payload"][0].numpy()], aggs)
    assert int(rows.item()) == len(rk[0])
    np.testing.assert_array_equal(ok[:len(rk[0])].cpu().numpy(), rk[0])


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

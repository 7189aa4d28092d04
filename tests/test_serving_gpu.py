"""Serving runtime on the GPU: every request's result in the mix (several
slots, continuous batching, overlapping calls) equals its result alone and
the oracle's; oversized requests are refused at submit; the footprint that
admission charges bounds the temporary bytes the path really uses."""
import ctypes

import numpy as np
import pytest
import torch

import datagen
import oracle
from paper_2010_00152_gb300 import sgagg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
AGG7 = [(0, 0), (1, 0), (2, 0), (3, 0), (1, 1), (2, 1), (3, 1)]


def to_np(t):
    return t.cpu().numpy()


def requests(count, seed, hi, key_dtype):
    out = []
    for r in datagen.config5_requests(count=count, seed=seed, hi=hi):
        c = datagen.config5_request(r, device=DEV)
        k = c["key_cols"][0]
        if key_dtype == torch.uint32:
            k = (k.view(torch.int64) & 0xFFFFFFFF).to(torch.uint32)
        out.append((k, c["payload"]))
    return out


@pytest.mark.parametrize("key_dtype", [torch.uint64, torch.uint32])
def test_served_equals_alone(key_dtype):
    reqs = requests(48, 3, 1 << 19, key_dtype)
    srv = sgagg.Server(AGG7, slots=4, device_budget_bytes=8 << 30, memory_budget_rows=1 << 16,
                       small_rows=1 << 15, max_batch=16, max_batch_rows=1 << 20)
    try:
        tickets = [srv.submit(k, p) for k, p in reqs]
        served = [srv.wait(t) for t in tickets]
    finally:
        srv.close()
    assert {s["status"] for s in served} == {0}
    assert max(s["batch_size"] for s in served) > 1  # some ran batched
    assert len({s["slot"] for s in served}) > 1       # several slots in use
    agg = sgagg.Aggregator(1 << 16)
    try:
        for i, ((k, p), s) in enumerate(zip(reqs, served)):
            ak, aa = agg.aggregate([k], p, AGG7)
            sk, sa = s["out"]
            assert s["rows"] == ak[0].numel()
            np.testing.assert_array_equal(to_np(sk), to_np(ak[0]))
            for j in range(len(AGG7)):
                np.testing.assert_array_equal(to_np(sa[j]), to_np(aa[j]))
            if i < 6:  # and the oracle, for a few
                rk, ra = oracle.aggregate([to_np(k)], [to_np(x) for x in p], AGG7)
                np.testing.assert_array_equal(to_np(sk), rk[0])
                for j in range(len(AGG7)):
                    np.testing.assert_array_equal(to_np(sa[j]), ra[j])
    finally:
        agg.close()


def test_plain_form_equals_served():
    reqs = requests(12, 5, 1 << 18, torch.uint64)
    res = {}
    for name, cfg in (("plain", dict(slots=1, small_rows=0)), ("served", dict(slots=3, small_rows=1 << 14))):
        srv = sgagg.Server(AGG7, device_budget_bytes=4 << 30, memory_budget_rows=1 << 15, max_batch=8,
                           max_batch_rows=1 << 20, **cfg)
        try:
            res[name] = [srv.wait(t) for t in [srv.submit(k, p) for k, p in reqs]]
        finally:
            srv.close()
    for a, b in zip(res["plain"], res["served"]):
        assert a["batch_size"] == 1 and a["slot"] == 0
        np.testing.assert_array_equal(to_np(a["out"][0]), to_np(b["out"][0]))
        for x, y in zip(a["out"][1], b["out"][1]):
            np.testing.assert_array_equal(to_np(x), to_np(y))


def test_capacity_error_stays_with_its_request():
    reqs = requests(6, 9, 1 << 13, torch.uint64)
    srv = sgagg.Server(AGG7, slots=2, device_budget_bytes=4 << 30, memory_budget_rows=1 << 15,
                       small_rows=1 << 14, max_batch=8, max_batch_rows=1 << 20)
    try:
        ts = [srv.submit(k, p, capacity=(1 if i == 2 else None)) for i, (k, p) in enumerate(reqs)]
        out = [srv.wait(t) for t in ts]
    finally:
        srv.close()
    distinct = [np.unique(to_np(k)).size for k, _ in reqs]
    for i, o in enumerate(out):
        if i == 2 and distinct[i] > 1:
            assert o["status"] == sgagg.SGAGG_ECAPACITY and o["rows"] == -1
        else:
            assert o["status"] == 0 and o["rows"] == distinct[i]


def test_oversized_request_refused_at_submit():
    srv = sgagg.Server(AGG7, slots=1, device_budget_bytes=1 << 30, memory_budget_rows=1 << 20)
    try:
        k = torch.zeros(8, dtype=torch.uint64, device=DEV)
        p = [torch.zeros(8, dtype=torch.int64, device=DEV)] * 2
        pay = (ctypes.c_void_p * 2)(*[x.data_ptr() for x in p])
        oa = (ctypes.c_void_p * 7)(*([k.data_ptr()] * 7))
        req = sgagg.sgagg_request(k.data_ptr(), 8, 2, ctypes.cast(pay, ctypes.c_void_p), 1 << 30, k.data_ptr(),
                                  ctypes.cast(oa, ctypes.c_void_p), 1 << 30, None)
        t = ctypes.c_int64(-7)
        st = sgagg.lib().sgagg_server_submit(srv.h, ctypes.byref(req), ctypes.byref(t))
        assert st == sgagg.SGAGG_ECAPACITY and t.value == -7
        # the server still serves
        r = srv.wait(srv.submit(k, p))
        assert r["status"] == 0 and r["rows"] == 1
    finally:
        srv.close()


@pytest.mark.parametrize("n,m", [(3000, 1 << 16), (200_000, 1 << 20), (1 << 20, 1 << 16)])
def test_footprint_bounds_temp_bytes(n, m):
    c = datagen.config5_request(dict(rows=n, D=max(1, n // 3), seed=11), device=DEV)
    agg = sgagg.Aggregator(m)
    try:
        agg.aggregate(c["key_cols"], c["payload"], AGG7)
        temp = agg.temp_bytes()
    finally:
        agg.close()
    fp = sgagg.sgagg_request_footprint(n, 8, 2, 7, n, m)
    assert temp <= fp - n * (8 + 16) - n * (8 + 56)

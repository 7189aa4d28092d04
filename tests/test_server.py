"""Serving runtime: admission and batching decisions (sgagg_server_simulate,
host only) and the footprint that admission charges.

The simulator runs the server's own scheduler against a cost model, so
these tests check the decisions the GPU server takes, without a GPU."""
import random

import pytest

from paper_2010_00152_gb300 import sgagg

N_PAYLOAD, N_AGGS = 2, 7


def footprint(n, m):
    # the closed form documented with sgagg_request_footprint, written out
    kb = 8
    inp = n * (kb + 8 * N_PAYLOAD)
    out = n * (kb + 8 * N_AGGS)
    b = min(n, m)
    ws = 8 * b * (3 + 3 * N_PAYLOAD + 3 * (1 + N_AGGS))
    runs = 8 * n * (1 + N_AGGS) if n > m else 0
    return inp + out + ws + runs + (64 << 20)


def test_footprint_closed_form():
    for n, m in [(0, 1), (1, 1 << 22), (1 << 20, 1 << 22), (1 << 24, 1 << 22), (12345, 100)]:
        assert sgagg.sgagg_request_footprint(n, 8, N_PAYLOAD, N_AGGS, n, m) == footprint(n, m)
    assert sgagg.sgagg_request_footprint(-1, 8, 1, 1, 0, 1) == -1


def workload(seed, count, lo=1 << 10, hi=1 << 22):
    rng = random.Random(seed)
    rows, arr, t = [], [], 0.0
    for _ in range(count):
        rows.append(int(lo * (hi / lo) ** rng.random()))
        t += rng.expovariate(1.0 / 300.0)
        arr.append(t)
    return rows, arr


def check_invariants(cfg, rows, arr, st, fi, sl, bt):
    n = len(rows)
    fps = [footprint(r, cfg.memory_budget_rows) for r in rows]
    admitted = [i for i in range(n) if sl[i] >= 0]
    for i in range(n):
        if sl[i] < 0:
            assert fps[i] > cfg.device_budget_bytes  # refused only when it can never fit
            assert bt[i] == -1
        else:
            assert fps[i] <= cfg.device_budget_bytes
            assert st[i] >= arr[i] - 1e-9 and fi[i] > st[i]
    # calls: members share start, finish and slot; batches hold small requests only
    calls = {}
    for i in admitted:
        calls.setdefault(bt[i], []).append(i)
    for b, mem in calls.items():
        assert len({(st[i], fi[i], sl[i]) for i in mem}) == 1
        if len(mem) > 1:  # batchable: small, and one chunk for 8-byte keys
            assert all(rows[i] <= min(cfg.small_rows, 8192) for i in mem)
            assert len(mem) <= cfg.max_batch
            assert sum(rows[i] for i in mem) <= cfg.max_batch_rows
        if any(rows[i] > min(cfg.small_rows, 8192) for i in mem):
            assert len(mem) == 1  # a request that cannot be batched runs alone
    # at every call start: slots and budget respected
    starts = sorted({st[mem[0]] for mem in calls.values()})
    for t in starts:
        live = [mem for mem in calls.values() if st[mem[0]] <= t < fi[mem[0]]]
        assert len(live) <= cfg.slots
        assert len({sl[mem[0]] for mem in live}) == len(live)  # one call per slot
        assert sum(fps[i] for mem in live for i in mem) <= cfg.device_budget_bytes
    # first come, first served: no admitted request starts before an earlier one
    order = sorted(admitted, key=lambda i: (arr[i], i))
    for a, b in zip(order, order[1:]):
        assert st[a] <= st[b] + 1e-9


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("slots,budget_gb,small", [(8, 64, 1 << 16), (2, 4, 1 << 14), (4, 1, 8192), (1, 64, 0)])
def test_scheduler_invariants(seed, slots, budget_gb, small):
    cfg = sgagg.server_config(slots=slots, device_budget_bytes=budget_gb << 30, memory_budget_rows=1 << 22,
                              small_rows=small, max_batch=32, max_batch_rows=1 << 20)
    rows, arr = workload(seed, 400)
    rows[5] = 1 << 36  # never fits
    res = sgagg.sgagg_server_simulate(cfg, N_PAYLOAD, N_AGGS, rows, arr, [50.0, 0.002, 3.0])
    check_invariants(cfg, rows, arr, *res)
    assert res[2][5] == -1


def test_plain_form_is_one_after_another():
    cfg = sgagg.server_config(slots=1, device_budget_bytes=64 << 30, memory_budget_rows=1 << 22, small_rows=0,
                              max_batch=1, max_batch_rows=1)
    rows, arr = workload(7, 200)
    cost = [40.0, 0.001, 2.0]
    st, fi, sl, bt = sgagg.sgagg_server_simulate(cfg, N_PAYLOAD, N_AGGS, rows, arr, cost)
    prev = 0.0
    for i in range(len(rows)):  # arrivals are increasing
        start = max(arr[i], prev)
        assert st[i] == pytest.approx(start)
        assert fi[i] == pytest.approx(start + cost[0] + cost[1] * rows[i] + cost[2])
        assert sl[i] == 0
        prev = fi[i]
    assert len(set(bt)) == len(rows)


def test_continuous_batching_joins_waiting_small_requests():
    # a burst of small requests while one slot is busy: the ones that arrive
    # during the first call run together as the next call
    cfg = sgagg.server_config(slots=1, device_budget_bytes=64 << 30, memory_budget_rows=1 << 22,
                              small_rows=1 << 16, max_batch=64, max_batch_rows=1 << 24)
    rows = [4096] * 20
    arr = [0.0] + [1.0 + i for i in range(19)]
    st, fi, sl, bt = sgagg.sgagg_server_simulate(cfg, N_PAYLOAD, N_AGGS, rows, arr, [100.0, 0.0, 1.0])
    assert bt[0] == 0 and st[0] == 0.0
    assert len(set(bt[1:])) == 1  # all 19 joined the second call
    assert st[1] == pytest.approx(fi[0])


def test_budget_blocks_until_release():
    # two requests that do not fit together run one after the other even
    # with free slots; the small one behind the big one waits (no overtaking)
    big = 1 << 24
    cfg = sgagg.server_config(slots=4, device_budget_bytes=footprint(big, 1 << 22) + 1,
                              memory_budget_rows=1 << 22, small_rows=1 << 16, max_batch=8, max_batch_rows=1 << 20)
    rows = [big, big, 1000]
    arr = [0.0, 1.0, 2.0]
    st, fi, sl, bt = sgagg.sgagg_server_simulate(cfg, N_PAYLOAD, N_AGGS, rows, arr, [10.0, 0.001, 0.0])
    assert st[1] == pytest.approx(fi[0])
    assert st[2] >= st[1]


def test_bad_config_rejected():
    cfg = sgagg.server_config(slots=0)
    with pytest.raises(sgagg.SgaggError):
        sgagg.sgagg_server_simulate(cfg, 1, 1, [1], [0.0], [1, 0, 0])

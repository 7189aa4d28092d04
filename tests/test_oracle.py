"""Pins for the CPU oracle (no GPU).

The oracle (sort + in-stream fold, plain C) is checked against things other
than itself:
  * a pure-Python O(n^2) grouper with a separate insertion sort of the group
    keys, on every n <= 64 over many seeds;
  * numpy's own routines where GROUP BY reduces to them (np.unique for the
    distinct keys and counts, ufunc.at for sums/min/max);
  * invariants every correct result has (strictly ascending keys, counts add
    up to n, sums preserve the input total mod 2^64, min/max are payload
    values of their key);
  * closed forms for the workloads (exactly 10,000 keys in the 2^20-row
    uniform workload; the 4-combination report workload).
Inputs mix negative payloads, keys with the top bit set, several payload
columns with aggregates over different columns, so that a dropped term, a
signed key comparison, swapped min/max or a transposed column fails.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle

MASK = (1 << 64) - 1


def to_s64(v):
    v &= MASK
    return v - (1 << 64) if v >= (1 << 63) else v


def brute_groupby(keys, payload, aggs):
    """O(n^2) grouping: each row scans the groups found so far."""
    gkeys, gstate = [], []
    for i in range(len(keys)):
        k = int(keys[i])
        hit = -1
        for g in range(len(gkeys)):
            if gkeys[g] == k:
                hit = g
                break
        vals = []
        for op, c in aggs:
            vals.append(1 if op == oracle.COUNT else int(payload[c][i]))
        if hit < 0:
            gkeys.append(k)
            gstate.append(list(vals))
        else:
            st = gstate[hit]
            for a, (op, c) in enumerate(aggs):
                if op in (oracle.COUNT, oracle.SUM):
                    st[a] = to_s64(st[a] + vals[a])
                elif op == oracle.MIN:
                    st[a] = min(st[a], vals[a])
                else:
                    st[a] = max(st[a], vals[a])
    # insertion sort of the groups by unsigned key
    order = []
    for g in range(len(gkeys)):
        j = len(order)
        order.append(g)
        while j > 0 and gkeys[order[j - 1]] > gkeys[order[j]]:
            order[j - 1], order[j] = order[j], order[j - 1]
            j -= 1
    return [gkeys[g] for g in order], [[gstate[g][a] for g in order] for a in range(len(aggs))]


AGGS3 = [(oracle.COUNT, 0), (oracle.SUM, 0), (oracle.MIN, 1), (oracle.MAX, 2),
         (oracle.SUM, 2), (oracle.MIN, 0), (oracle.MAX, 1)]


def small_case(n, seed):
    rng = np.random.default_rng(seed)
    dom = int(rng.integers(1, max(2, n) + 2))
    base = rng.integers(0, 2**64, size=dom, dtype=np.uint64)
    keys = base[rng.integers(0, dom, size=n)]
    pay = [rng.integers(-2**63, 2**63, size=n, dtype=np.int64) if c == 0 else
           rng.integers(-50, 50, size=n).astype(np.int64) for c in range(3)]
    return keys, pay


@pytest.mark.parametrize("n", list(range(0, 65)))
def test_oracle_matches_bruteforce(n):
    for seed in range(6):
        keys, pay = small_case(n, 1000 * n + seed)
        ok, oa = oracle.groupby(keys, pay, AGGS3)
        bk, ba = brute_groupby(keys, pay, AGGS3)
        assert [int(x) for x in ok] == bk
        for a in range(len(AGGS3)):
            assert [int(x) for x in oa[a]] == ba[a], (n, seed, a)


def numpy_groupby(keys, payload, aggs):
    """GROUP BY through numpy's library routines."""
    uk, inv, cnt = np.unique(keys, return_inverse=True, return_counts=True)
    out = []
    for op, c in aggs:
        if op == oracle.COUNT:
            out.append(cnt.astype(np.int64))
        elif op == oracle.SUM:
            s = np.zeros(len(uk), dtype=np.uint64)
            np.add.at(s, inv, payload[c].view(np.uint64))
            out.append(s.view(np.int64))
        elif op == oracle.MIN:
            m = np.full(len(uk), np.iinfo(np.int64).max, dtype=np.int64)
            np.minimum.at(m, inv, payload[c])
            out.append(m)
        else:
            m = np.full(len(uk), np.iinfo(np.int64).min, dtype=np.int64)
            np.maximum.at(m, inv, payload[c])
            out.append(m)
    return uk, out


@pytest.mark.parametrize("kind", ["c1", "wide", "extremes", "all_equal", "sorted", "reverse",
                                  "same_digit", "small_int", "clustered", "heavy_light"])
def test_oracle_matches_numpy(kind):
    n = 200_003
    if kind == "c1":
        c = datagen.config1(n=n, seed=3)
        keys = c["key_cols"][0].numpy()
        pay = [c["payload"][0].numpy(), datagen.uniform_int(3, 77, n, -10**6, 10**6).numpy(),
               datagen.rand64(3, 78, n).numpy()]
    elif kind == "wide":
        keys = datagen.keys_uniform_over(5, 1, n, 1 << 40).view(torch.uint64).numpy()
        pay = [datagen.rand64(5, c, n).numpy() for c in range(3)]
    else:
        keys = datagen.edge_keys(kind, n).numpy()
        pay = [datagen.rand64(9, c, n).numpy() for c in range(3)]
    ok, oa = oracle.groupby(keys, pay, AGGS3)
    uk, ua = numpy_groupby(keys, pay, AGGS3)
    np.testing.assert_array_equal(ok, uk)
    for a in range(len(AGGS3)):
        np.testing.assert_array_equal(oa[a], ua[a])


def check_invariants(keys, payload, aggs, ok, oa):
    n = len(keys)
    assert np.all(ok[1:] > ok[:-1]), "keys strictly ascending (unsigned)"
    assert len(ok) == len(np.unique(keys))
    for a, (op, c) in enumerate(aggs):
        if op == oracle.COUNT:
            assert int(oa[a].sum()) == n
            assert np.all(oa[a] >= 1)
        elif op == oracle.SUM:
            tot = int(payload[c].view(np.uint64).sum(dtype=np.uint64))
            got = int(oa[a].view(np.uint64).sum(dtype=np.uint64))
            assert tot == got
    # min <= max and both are payload values of that key
    mins = [(a, c) for a, (op, c) in enumerate(aggs) if op == oracle.MIN]
    maxs = {c: a for a, (op, c) in enumerate(aggs) if op == oracle.MAX}
    order = np.argsort(keys, kind="stable")
    sk = keys[order]
    starts = np.searchsorted(sk, ok, side="left")
    ends = np.searchsorted(sk, ok, side="right")
    for a, c in mins:
        vals = payload[c][order]
        for g in range(0, len(ok), max(1, len(ok) // 200)):
            seg = vals[starts[g]:ends[g]]
            assert oa[a][g] in seg
            if c in maxs:
                assert oa[a][g] <= oa[maxs[c]][g]
                assert oa[maxs[c]][g] in seg


def test_invariants_c1_full_size():
    c = datagen.config1()  # 2^20 rows, 10,000-value domain
    keys = c["key_cols"][0].numpy()
    pay = [p.numpy() for p in c["payload"]]
    ok, oa = oracle.groupby(keys, pay, c["aggs"])
    # every one of the 10,000 values occurs (P(some value missing) ~ 1e4 * e^-105)
    assert len(ok) == 10_000
    check_invariants(keys, pay, c["aggs"], ok, oa)


def test_c2_report_shape_closed_form():
    n = 1 << 18
    c = datagen.config2(n=n, seed=2)
    kc = [x.numpy() for x in c["key_cols"]]
    pay = [p.numpy() for p in c["payload"]]
    outk, oa = oracle.aggregate(kc, pay, c["aggs"])
    combos = list(zip([int(x) for x in outk[0]], [int(x) for x in outk[1]]))
    assert combos == sorted(datagen.C2_COMBOS)
    # direct per-combination accumulation: four accumulators
    sel = np.full(n, -1)
    for i, (a, b) in enumerate(combos):
        sel[(kc[0] == a) & (kc[1] == b)] = i
    assert np.all(sel >= 0)
    cnt = np.bincount(sel, minlength=4)
    np.testing.assert_array_equal(oa[0], cnt)
    assert abs(cnt[0] / n - 0.49) < 0.01 and abs(cnt[3] / n - 0.02) < 0.005
    for col in range(4):
        for i in range(4):
            v = pay[col][sel == i]
            assert oa[1 + 3 * col][i] == int(v.sum())
            assert oa[2 + 3 * col][i] == int(v.min())
            assert oa[3 + 3 * col][i] == int(v.max())


def test_normalized_key_order_is_lexicographic():
    rng = np.random.default_rng(4)
    n = 5000
    widths = [1, 2, 1, 4]
    cols = [rng.integers(0, 2 ** (8 * w), size=n, dtype=np.uint64).astype(
        {1: np.uint8, 2: np.uint16, 4: np.uint32}[w]) for w in widths]
    keys = oracle.normalize(cols)
    tuples = list(zip(*[[int(x) for x in c] for c in cols]))
    by_tuple = sorted(range(n), key=lambda i: (tuples[i], i))
    by_key = sorted(range(n), key=lambda i: (int(keys[i]), i))
    assert by_tuple == by_key
    for c in range(len(widths)):
        np.testing.assert_array_equal(oracle.unpack(keys, widths, c), cols[c])


def test_normalize_rejects_too_wide():
    with pytest.raises(ValueError):
        oracle.normalize([np.zeros(3, np.uint64), np.zeros(3, np.uint8)])


def test_wraparound_sums():
    keys = np.array([5, 5, 5, 9], dtype=np.uint64)
    big = np.iinfo(np.int64).max
    pay = [np.array([big, big, 3, np.iinfo(np.int64).min], dtype=np.int64)]
    ok, oa = oracle.groupby(keys, pay, [(oracle.SUM, 0), (oracle.MIN, 0), (oracle.MAX, 0)])
    assert list(ok) == [5, 9]
    assert int(oa[0][0]) == to_s64(2 * big + 3)
    assert int(oa[1][0]) == 3 and int(oa[2][0]) == big


@pytest.mark.parametrize("M", [1, 7, 64, 1000, 65_536, 10**9])
def test_runs_fold_back_to_groupby(M):
    """Merging the early-aggregated runs gives the plain result for any memory
    budget (the method is exact), and each run is its batch's distinct keys."""
    n = 20_000 if M > 1 else 3000
    c = datagen.config1(n=n, seed=11, D=1500)
    keys = c["key_cols"][0].numpy()
    pay = [c["payload"][0].numpy()]
    rows, rk, rs = oracle.run_generation(keys, pay, c["aggs"], M)
    assert len(rows) == -(-n // M)
    for b, r in enumerate(rows):
        assert r == len(np.unique(keys[b * M:(b + 1) * M]))
    fk, fa = oracle.fold_states(rk, rs, [op for op, _ in c["aggs"]])
    ok, oa = oracle.groupby(keys, pay, c["aggs"])
    np.testing.assert_array_equal(fk, ok)
    for a in range(len(oa)):
        np.testing.assert_array_equal(fa[a], oa[a])


def test_bad_spec_rejected():
    with pytest.raises(ValueError):
        oracle.groupby(np.zeros(3, np.uint64), [np.zeros(3, np.int64)], [(oracle.SUM, 1)])
    with pytest.raises(ValueError):
        oracle.groupby(np.zeros(3, np.uint64), [np.zeros(3, np.int64)], [(7, 0)])

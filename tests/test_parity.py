"""GPU path vs the CPU oracle, element by element (bit-exact: int64 results).

Every case calls the CUDA library through the C ABI (binding in
paper_2010_00152_gb300/sgagg.py) on seeded inputs and compares keys and every
aggregate with the oracle.  Sizes span many chunks and ragged tails; edge
cases cover empty/tiny inputs, tile and budget boundaries, one key, all keys
distinct, extreme keys and payloads, adversarial key layouts, composite keys,
every key width, the pre-fold switch, the pinned-host run arena and the
capacity error.
"""
import numpy as np
import pytest
import torch

import datagen
import oracle
from paper_2010_00152_gb300 import sgagg

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TILE = 8192


def to_np(t):
    return t.cpu().numpy()


def gpu_run(key_cols, payload, aggs, M, capacity=None, **opts):
    agg = sgagg.Aggregator(M, **opts)
    try:
        kc = [k.to(DEV) for k in key_cols]
        pc = [p.to(DEV) for p in payload]
        ok, oa = agg.aggregate(kc, pc, aggs, capacity=capacity)
        st = agg.stats()
        tb = agg.temp_bytes()
        return [to_np(k) for k in ok], [to_np(a) for a in oa], st, tb
    finally:
        agg.close()


def oracle_run(key_cols, payload, aggs):
    return oracle.aggregate([to_np(k) for k in key_cols], [to_np(p) for p in payload], aggs)


def check(key_cols, payload, aggs, M, **opts):
    gk, ga, st, tb = gpu_run(key_cols, payload, aggs, M, **opts)
    rk, ra = oracle_run(key_cols, payload, aggs)
    assert len(gk[0]) == len(rk[0]), (len(gk[0]), len(rk[0]))
    for c in range(len(rk)):
        np.testing.assert_array_equal(gk[c], rk[c])
    for a in range(len(ra)):
        np.testing.assert_array_equal(ga[a], ra[a], err_msg="aggregate %d" % a)
    return st, tb


AGG4 = [(0, 0), (1, 0), (2, 0), (3, 0)]


def u64_case(kind, n, seed=3, npay=1):
    keys = datagen.edge_keys(kind, n, seed) if kind not in ("c1",) else \
        datagen.config1(n=n, seed=seed)["key_cols"][0]
    pay = [datagen.uniform_int(seed, 20 + c, n, -10**12, 10**12) for c in range(npay)]
    return [keys], pay


@pytest.mark.parametrize("n", [0, 1, 2, 31, 32, 33, TILE - 1, TILE, TILE + 1, 3 * TILE + 17, 100_003])
def test_sizes_single_batch(n):
    kc, pay = u64_case("c1", n)
    check(kc, pay, AGG4, M=1 << 30)


@pytest.mark.parametrize("M", [TILE - 1, TILE, TILE + 1, 10_000, 65_536, 99_999])
def test_budget_boundaries(M):
    kc, pay = u64_case("c1", 200_003)
    st, _ = check(kc, pay, AGG4, M=M)
    B = -(-200_003 // M)
    assert st["batches"] == B
    assert st["runs"] == (B if B > 1 else 0)


def test_budget_one_row():
    """300 one-row runs exceed one merge's fan-in (256): one preliminary merge
    of the 45 smallest runs writes one more run (counted in the spill)."""
    kc, pay = u64_case("c1", 300)
    st, _ = check(kc, pay, AGG4, M=1)
    assert st["batches"] == 300 and st["runs"] == 301 and st["run_rows"] == 300 + 45


def test_budget_not_dividing_n():
    kc, pay = u64_case("c1", 123_457)
    check(kc, pay, AGG4, M=40_000)


@pytest.mark.parametrize("kind", ["all_equal", "distinct", "sorted", "reverse", "small_int",
                                  "extremes", "same_digit", "clustered", "heavy_light"])
@pytest.mark.parametrize("M", [1 << 30, 50_000])
def test_adversarial_keys(kind, M):
    kc, pay = u64_case(kind, 150_001, npay=2)
    aggs = [(0, 0), (1, 0), (2, 1), (3, 1), (1, 1), (2, 0), (3, 0)]
    check(kc, pay, aggs, M=M)


def test_payload_extremes_wraparound():
    n = 70_000
    keys = datagen.keys_uniform_over(9, 1, n, 50).view(torch.uint64)
    r = datagen.uniform_int(9, 2, n, 0, 3)
    vals = torch.tensor([np.iinfo(np.int64).max, np.iinfo(np.int64).min, -1, 0], dtype=torch.int64)
    pay = [vals[r]]
    check([keys], pay, AGG4, M=1 << 30)
    check([keys], pay, AGG4, M=9_000)


def test_c1_full_size_and_run_rows():
    """Config 1 at full size: 2^20 rows, 10,000 keys, 16 runs + wide merge.
    The run bookkeeping equals the oracle's run generation exactly."""
    c = datagen.config1()
    st, tb = check(c["key_cols"], c["payload"], c["aggs"], M=c["M"])
    rows, _, _ = oracle.run_generation(to_np(c["key_cols"][0]), [to_np(c["payload"][0])],
                                       c["aggs"], c["M"])
    assert st["runs"] == 16 and st["run_rows"] == sum(rows)
    assert st["out_rows"] == 10_000
    assert tb >= st["run_rows"] * 8 * (1 + len(c["aggs"]))


@pytest.mark.parametrize("one_pass", [1, 0])
@pytest.mark.parametrize("shape", [(1 << 20, 10_000, 65_536), (300_001, 200_000, 20_000)])
def test_runs_one_pass_or_batch_at_a_time(one_pass, shape):
    """Small batches: the runs of all batches generated in one pass per step
    (the default here) or one batch at a time.  Same output as the oracle,
    and every run's row count, in order, equals the oracle's run generation
    (Sec. 3: each run holds its batch's distinct keys once)."""
    n, D, M = shape
    c = datagen.config1(n=n, seed=17, D=D, M=M)
    agg = sgagg.Aggregator(M, one_pass=one_pass)
    try:
        ok, oa = agg.aggregate([c["key_cols"][0].to(DEV)], [c["payload"][0].to(DEV)], c["aggs"])
        st = agg.stats()
        sizes = list(agg.run_sizes())
    finally:
        agg.close()
    assert st["one_pass"] == one_pass
    rk, ra = oracle_run(c["key_cols"], c["payload"], c["aggs"])
    np.testing.assert_array_equal(to_np(ok[0]), rk[0])
    for a in range(len(ra)):
        np.testing.assert_array_equal(to_np(oa[a]), ra[a])
    rows, _, _ = oracle.run_generation(to_np(c["key_cols"][0]), [to_np(c["payload"][0])], c["aggs"], M)
    assert sizes == [int(r) for r in rows]


@pytest.mark.parametrize("opts", [dict(), dict(fanin_cap=4)])
def test_runs_one_pass_composite_key(opts):
    """A composite key of two 16-bit columns over 8 batches of 40,000 rows:
    all runs in one pass, then one wide merge (or preliminary merges of at
    most 4 runs first).  Same output as the oracle."""
    n = 320_000
    k0 = datagen.uniform_int(41, 1, n, 0, 300).to(torch.int64).to(torch.uint16)
    k1 = datagen.uniform_int(41, 2, n, 0, 999).to(torch.int64).to(torch.uint16)
    pay = [datagen.uniform_int(41, 3, n, -10**9, 10**9)]
    st, _ = check([k0, k1], pay, AGG4, M=40_000, prefold=0, **opts)
    # 8 runs from the batches; with the fan-in cap, preliminary merges write more
    assert st["one_pass"] == 1 and (st["runs"] == 8 if not opts else st["runs"] > 8)


def test_c2_report_shape_prefold():
    c = datagen.config2(n=1 << 22, seed=2)
    st, _ = check(c["key_cols"], c["payload"], c["aggs"], M=c["M"], lowcard=0)
    assert st["out_rows"] == 4 and st["prefold_passes"] >= 1


def test_c2_report_shape_streaming():
    """Four key combinations in one batch: one streaming fold (no sort)."""
    c = datagen.config2(n=1 << 22, seed=3)
    st, _ = check(c["key_cols"], c["payload"], c["aggs"], M=c["M"])
    assert st["out_rows"] == 4 and st["kernels"]["stream"]["launches"] == 2
    assert st["prefold_passes"] == 0 and st["kernel_launches"] <= 4


@pytest.mark.parametrize("nkeys", [1, 2, 7, 16, 17])
@pytest.mark.parametrize("n", [1 << 16, 300_007])
def test_few_keys_streaming_or_general(nkeys, n):
    """Up to 16 distinct keys take the streaming fold, 17 the sort; both give
    the oracle's result, with every aggregate kind on two payloads."""
    vals = datagen.uniform_int(31, 1, nkeys, 0, (1 << 62))
    r = datagen.uniform_int(31, 2, n, 0, nkeys - 1)
    keys = vals[r].view(torch.uint64)
    pay = [datagen.uniform_int(31, 3, n, -10**15, 10**15), datagen.uniform_int(31, 4, n, -5, 5)]
    aggs = [(0, 0), (1, 0), (2, 0), (3, 0), (1, 1), (2, 1), (3, 1)]
    st, _ = check([keys], pay, aggs, M=1 << 30)
    streamed = st["kernels"]["stream"]["launches"] > 0
    kd = len(np.unique(keys.numpy()))
    assert streamed == (kd <= 16 and kd * len(aggs) <= 104)  # accumulators per thread


def test_few_keys_sample_misses_a_key():
    """A key the planner's sample does not see (one row, off the sampled
    positions) makes the streaming fold give up; the general path groups the
    input and the result is exact."""
    n = 1 << 17  # the sample reads rows i * n / 16384, multiples of 8
    keys = torch.tensor([11, 22, 33], dtype=torch.int64)[datagen.uniform_int(5, 1, n, 0, 2)]
    keys[12_345] = 99  # an odd row: never sampled
    pay = [datagen.uniform_int(5, 2, n, -1000, 1000)]
    st, _ = check([keys.view(torch.uint64)], pay, AGG4, M=1 << 30)
    assert st["out_rows"] == 4 and st["split_segments"] >= 1


def test_c3_shape_reduced():
    c = datagen.config3(n=1 << 22, seed=1, D=1 << 21, M=1 << 18)
    st, _ = check(c["key_cols"], c["payload"], c["aggs"], M=c["M"])
    rows, _, _ = oracle.run_generation(to_np(c["key_cols"][0]), [to_np(c["payload"][0])],
                                       c["aggs"], c["M"])
    assert st["runs"] == 16 and st["run_rows"] == sum(rows)


@pytest.mark.parametrize("mask", [-1, 1 << sgagg.KERNEL_CLASSES.index("merge"), 0])
def test_timing_classes(mask):
    """Per-launch CUDA-event timing of some kernel classes only: the result
    is the oracle's, timed classes report time, the others none, and every
    launch is still counted."""
    c = datagen.config3(n=1 << 21, seed=2, D=1 << 20, M=1 << 17)
    st, _ = check(c["key_cols"], c["payload"], c["aggs"], M=c["M"], timing=1, timing_classes=mask)
    k = st["kernels"]
    for i, name in enumerate(sgagg.KERNEL_CLASSES):
        if k[name]["launches"] == 0:
            continue
        assert (k[name]["ms"] > 0) == bool((mask >> i) & 1), (name, k[name])
    assert k["merge"]["launches"] == 3 and k["rungen"]["launches"] >= 1
    assert st["kernel_launches"] == sum(v["launches"] for v in k.values())


@pytest.mark.parametrize("widths", [[1], [2], [4], [8], [1, 1], [2, 4], [1, 2, 1], [4, 4], [1, 1, 1, 1, 1, 1, 1, 1]])
def test_composite_keys(widths):
    n = 120_000
    dt = {1: torch.uint8, 2: torch.uint16, 4: torch.uint32, 8: torch.uint64}
    cols = []
    for i, w in enumerate(widths):
        hi = min((1 << (8 * w)) - 1, 40 if len(widths) > 1 else (1 << 62))
        v = datagen.uniform_int(11, 30 + i, n, 0, hi)
        cols.append(v.to(dt[w]) if w < 8 else v.view(torch.uint64))
    pay = [datagen.uniform_int(11, 50, n, -100, 100)]
    check(cols, pay, AGG4, M=1 << 30)
    check(cols, pay, AGG4, M=30_000)


def test_c4_instance_shape():
    inst = dict(rows=300_000, D=5000, seed=17)
    c = datagen.config4_instance(inst)
    check(c["key_cols"], c["payload"], c["aggs"], M=c["M"])


def test_c5_request_shape():
    req = dict(rows=500_000, D=700, seed=23)
    c = datagen.config5_request(req, M=1 << 17)
    check(c["key_cols"], c["payload"], c["aggs"], M=c["M"])


@pytest.mark.parametrize("prefold", [0, 1])
def test_prefold_switch_invariant(prefold):
    c = datagen.config1(n=300_000, seed=8, D=20_000)
    check(c["key_cols"], c["payload"], c["aggs"], M=100_000, prefold=prefold)


@pytest.mark.parametrize("aggs", [
    [(3, 0), (1, 0), (0, 0), (2, 0)],                  # max, sum, count, min: the pattern out of order
    [(1, 0), (2, 0), (3, 0), (1, 0)],                  # a repeated sum: not the pattern
    [(2, 1), (1, 0), (3, 1), (2, 0), (1, 1), (3, 0)],  # the pattern on two columns, interleaved
])
@pytest.mark.parametrize("n, D", [(8191, 8000), (60_000, 2000), (70_000, 7)])
def test_aggregate_orders(aggs, n, D):
    """Sum, min and max of one column are folded in one pass when they are
    exactly that triple: each result must land in its own output column
    whatever the aggregates' order, and other lists take the per-aggregate
    fold.  Sizes cover one-row groups (a lane per group), small groups
    (segmented scans) and a few large groups."""
    c = datagen.config1(n=n, seed=31, D=D)
    pay = [c["payload"][0], datagen.uniform_int(31, 7, n, -10**15, 10**15)]
    check(c["key_cols"], pay, aggs, M=1 << 30)
    check(c["key_cols"], pay, aggs, M=max(1, n // 5))


@pytest.mark.parametrize("bins", [0, 1])
def test_prefold_bins_invariant(bins):
    """Tile pre-aggregation binned by key range or by a hash of the key, on
    Zipf ranks used as keys (the frequent keys crowd the low end of the
    range, so range bins there hold many keys): same result."""
    n = 200_000
    keys = datagen.zipf_ranks(21, 1, n, 300_000).to(torch.int64).view(torch.uint64)
    pay = [datagen.uniform_int(21, 2, n, -1000, 1000)]
    aggs = [(0, 0), (1, 0), (2, 0), (3, 0)]
    st, _ = check([keys], pay, aggs, M=100_000, prefold=1, prefold_bins=bins)
    assert st["prefold_passes"] >= 1


@pytest.mark.parametrize("bits", [0, 9, 15])
def test_single_level_partition(bits):
    """Every row written once to its final bucket (no second partition
    level), at the automatic and at wide digits: same result."""
    c = datagen.config1(n=300_000, seed=19, D=200_000)
    check(c["key_cols"], c["payload"], c["aggs"], M=150_000, radix_bits=bits, part_levels=1)


@pytest.mark.parametrize("bits", [1, 4, 9, 15])
def test_radix_bits_invariant(bits):
    c = datagen.config1(n=300_000, seed=8, D=200_000)
    check(c["key_cols"], c["payload"], c["aggs"], M=150_000, radix_bits=bits)


def test_runs_spill_to_pinned_host():
    c = datagen.config1(n=400_000, seed=4, D=150_000)
    st, _ = check(c["key_cols"], c["payload"], c["aggs"], M=50_000, arena_cap=3 * 50_000 * 40)
    assert st["run_bytes_host"] > 0 and st["run_bytes_device"] > 0


def test_permutation_invariance():
    c = datagen.config1(n=200_000, seed=12, D=30_000)
    perm = torch.randperm(200_000, generator=torch.Generator().manual_seed(5))
    a = gpu_run(c["key_cols"], c["payload"], c["aggs"], 60_000)
    pk = c["key_cols"][0].view(torch.int64)[perm].view(torch.uint64)
    b = gpu_run([pk], [c["payload"][0][perm]], c["aggs"], 60_000)
    for x, y in zip(a[0] + a[1], b[0] + b[1]):
        np.testing.assert_array_equal(x, y)


def test_capacity_error():
    c = datagen.config1(n=50_000, seed=2, D=1000)
    with pytest.raises(sgagg.SgaggError) as e:
        gpu_run(c["key_cols"], c["payload"], c["aggs"], 1 << 30, capacity=500)
    assert e.value.status == sgagg.SGAGG_ECAPACITY
    with pytest.raises(sgagg.SgaggError) as e:
        gpu_run(c["key_cols"], c["payload"], c["aggs"], 10_000, capacity=500)
    assert e.value.status == sgagg.SGAGG_ECAPACITY


def test_host_buffers_entry_point():
    c = datagen.config1(n=150_000, seed=6, D=7_000)
    agg = sgagg.Aggregator(40_000)
    try:
        ok, oa = agg.aggregate_host([to_np(c["key_cols"][0])], [to_np(c["payload"][0])], c["aggs"])
    finally:
        agg.close()
    rk, ra = oracle_run(c["key_cols"], c["payload"], c["aggs"])
    np.testing.assert_array_equal(ok[0], rk[0])
    for a in range(len(ra)):
        np.testing.assert_array_equal(oa[a], ra[a])


@pytest.mark.parametrize("case", ["batches", "one_batch", "composite", "absorbing", "empty", "many_parts",
                                  "pinned"])
def test_host_buffers_staged(case):
    """Host-buffer calls copy the input batch by batch and the merged output
    back in parts; every layout gives the oracle's result."""
    aggs = [(0, 0), (1, 0), (2, 1), (3, 1)]
    opts, M = {}, 30_000
    if case == "composite":
        c = datagen.config2(n=120_000)
        kc = [to_np(k) for k in c["key_cols"]]
        pc = [to_np(p) for p in c["payload"]]
        aggs, M = c["aggs"], 7_000
    else:
        n = {"batches": 200_003, "one_batch": 20_000, "absorbing": 150_000, "empty": 0,
             "many_parts": 400_000, "pinned": 123_457}[case]
        c = datagen.config5_request(dict(rows=n, D=max(1, n // 3), seed=17), M=M)
        kc = [to_np(c["key_cols"][0])]
        pc = [to_np(p) for p in c["payload"]]
        if case == "absorbing":
            opts = dict(policy=1, absorb_batch=11_000)
        if case == "many_parts":
            M = 9_000
    if case == "pinned":
        kc = [torch.from_numpy(k).pin_memory().numpy() for k in kc]
        pc = [torch.from_numpy(p).pin_memory().numpy() for p in pc]
    agg = sgagg.Aggregator(M, **opts)
    try:
        ok, oa = agg.aggregate_host(kc, pc, aggs)
    finally:
        agg.close()
    rk, ra = oracle.aggregate(kc, pc, aggs)
    for a, b in zip(ok, rk):
        np.testing.assert_array_equal(a, b)
    for a, b in zip(oa, ra):
        np.testing.assert_array_equal(a, b)


def test_handle_reuse_across_shapes():
    agg = sgagg.Aggregator(30_000)
    try:
        for seed, n, D in ((1, 100_000, 500), (2, 7, 3), (3, 90_001, 80_000), (4, 0, 1)):
            c = datagen.config1(n=n, seed=seed, D=D)
            kc = [c["key_cols"][0].to(DEV)]
            pc = [c["payload"][0].to(DEV)]
            ok, oa = agg.aggregate(kc, pc, c["aggs"])
            rk, ra = oracle_run(c["key_cols"], c["payload"], c["aggs"])
            np.testing.assert_array_equal(to_np(ok[0]), rk[0])
            for a in range(len(ra)):
                np.testing.assert_array_equal(to_np(oa[a]), ra[a])
    finally:
        agg.close()


def test_merge_big_groups():
    """~100 runs that each hold nearly every one of 500 keys: merge tiles of
    some 80 key groups of ~100 rows each (groups across scan windows)."""
    c = datagen.config1(n=200_003, seed=17, D=500)
    st, _ = check(c["key_cols"], c["payload"], c["aggs"], M=2048)
    assert st["runs"] == 98


@pytest.mark.parametrize("cap", [2, 3, 7])
def test_preliminary_merges(cap):
    """More runs than one wide merge may take: the smallest runs are merged
    first (Sec. 4.3) until the final merge takes them all."""
    c = datagen.config1(n=60_000, seed=13, D=9000)
    st, _ = check(c["key_cols"], c["payload"], c["aggs"], M=1000, fanin_cap=cap)
    assert st["runs"] > 60


def _batched_case(seed, sizes, domains, key_dtype=torch.uint32):
    insts = []
    for i, (n, D) in enumerate(zip(sizes, domains)):
        c = datagen.config4_instance(dict(rows=n, D=D, seed=seed * 1000 + i)) if n > 0 else None
        if c is None:
            k = torch.empty(0, dtype=key_dtype)
            p = torch.empty(0, dtype=torch.int64)
        else:
            k = c["key_cols"][0]
            p = c["payload"][0]
            if key_dtype != torch.uint32:
                k = k.to(torch.int64).to(key_dtype) if key_dtype != torch.uint64 else k.to(torch.int64).view(torch.uint64)
        insts.append((k, [p]))
    return insts


@pytest.mark.parametrize("key_dtype", [torch.uint32, torch.uint16, torch.uint64])
def test_batched_matches_oracle(key_dtype):
    """Independent instances of uneven sizes in one batched call; every
    instance equals its own oracle result."""
    sizes = [0, 1, 5, 1000, 8192, 8193, 20_000, 70_001, 3, 150_000, 9000, 12]
    domains = [1, 1, 3, 16, 500, 20_000, 5, 100_000, 2, 1_000, 60_000, 7]
    insts = _batched_case(3, sizes, domains, key_dtype)
    aggs = [(0, 0), (1, 0), (2, 0), (3, 0)]
    agg = sgagg.Aggregator(1 << 20)
    try:
        res = agg.aggregate_batched([(k.to(DEV), [p.to(DEV) for p in pay]) for k, pay in insts], aggs)
        st = agg.stats()
    finally:
        agg.close()
    assert st["n_rows"] == sum(sizes)
    for (k, pay), r in zip(insts, res):
        rk, ra = oracle_run([k], pay, aggs)
        assert r is not None
        np.testing.assert_array_equal(to_np(r[0]), rk[0])
        for a in range(len(aggs)):
            np.testing.assert_array_equal(to_np(r[1][a]), ra[a])


@pytest.mark.parametrize("opts", [dict(prefold_bins=1), dict(prefold_rows=1024), dict(prefold_rows=3000),
                                  dict(batch_group_rows=1 << 16), dict(batch_group_rows=1 << 20)])
def test_batched_prefold_options(opts):
    """The batched call with hash-binned or smaller pre-aggregation tiles, or
    its instances grouped in smaller or bigger passes: every instance still
    equals its own oracle result."""
    sizes = [8193, 20_000, 70_001, 150_000, 9000]
    domains = [20_000, 5, 100_000, 1_000_000, 60_000]
    insts = _batched_case(4, sizes, domains)
    aggs = [(0, 0), (1, 0), (2, 0), (3, 0)]
    agg = sgagg.Aggregator(1 << 20, **opts)
    try:
        res = agg.aggregate_batched([(k.to(DEV), [p.to(DEV) for p in pay]) for k, pay in insts], aggs)
    finally:
        agg.close()
    for (k, pay), r in zip(insts, res):
        rk, ra = oracle_run([k], pay, aggs)
        np.testing.assert_array_equal(to_np(r[0]), rk[0])
        for j in range(len(aggs)):
            np.testing.assert_array_equal(to_np(r[1][j]), ra[j])


def test_batched_autotune(tmp_path):
    """Aggregator(autotune=True) sets the options a cache gives for the
    call's shape: here instance groups of 2^16 rows, seen as one
    pre-aggregation pass per group.  Same results as the oracle."""
    from paper_2010_00152_gb300 import tuning
    sizes = [8193, 20_000, 70_001, 150_000, 9000]
    domains = [20_000, 5, 100_000, 1_000_000, 60_000]
    insts = _batched_case(6, sizes, domains)
    aggs = [(0, 0), (1, 0), (2, 0), (3, 0)]
    cache = {}
    key = tuning.shape_key("batched", sum(sizes), 32, len(aggs))
    for d in range(4):  # whatever duplicate share the first call measures
        tuning.record(cache, key + "|d%d" % d, [({"batch_group_rows": 1 << 16}, 1.0)], "test")
    path = tmp_path / "tuning.json"
    tuning.save(cache, str(path))
    agg = sgagg.Aggregator(1 << 20, autotune=True, cache=str(path))
    try:
        for _ in range(2):
            res = agg.aggregate_batched([(k.to(DEV), [p.to(DEV) for p in pay]) for k, pay in insts], aggs)
            for (k, pay), r in zip(insts, res):
                rk, ra = oracle_run([k], pay, aggs)
                np.testing.assert_array_equal(to_np(r[0]), rk[0])
                for j in range(len(aggs)):
                    np.testing.assert_array_equal(to_np(r[1][j]), ra[j])
        st = agg.stats()
        chosen = agg.last_autotune
    finally:
        agg.close()
    assert chosen["options"] == {"batch_group_rows": 1 << 16}, chosen
    assert chosen["source"] in ("cache", "nearest")
    assert st["prefold_passes"] > 1


def test_batched_clustered_instances():
    """Instances whose keys crowd one end of their range (one bucket of the
    per-instance digit far above a chunk), one key value, and a wide spread;
    every instance equals its own oracle result."""
    g = torch.Generator().manual_seed(11)
    a = torch.cat([torch.randperm(40_000, generator=g), torch.tensor([2**32 - 1, 2**32 - 2, 2**31])])
    b = torch.full((50_000,), 7)
    c = torch.randint(0, 2**32, (60_000,), generator=g)
    d = torch.randint(0, 20, (9_000,), generator=g)
    insts = []
    for k in (a, b, c, d):
        k = k.to(torch.int64).to(torch.uint32)
        p = torch.randint(-1000, 1001, (k.numel(),), generator=g, dtype=torch.int64)
        insts.append((k, [p]))
    aggs = [(0, 0), (1, 0), (2, 0), (3, 0)]
    agg = sgagg.Aggregator(1 << 20)
    try:
        res = agg.aggregate_batched([(k.to(DEV), [p.to(DEV) for p in pay]) for k, pay in insts], aggs)
    finally:
        agg.close()
    for (k, pay), r in zip(insts, res):
        rk, ra = oracle_run([k], pay, aggs)
        np.testing.assert_array_equal(to_np(r[0]), rk[0])
        for j in range(len(aggs)):
            np.testing.assert_array_equal(to_np(r[1][j]), ra[j])


def test_batched_capacity_and_equals_plain():
    insts = _batched_case(5, [4000, 30_000, 100], [4000, 200, 100])
    aggs = [(0, 0), (1, 0), (2, 0)]
    agg = sgagg.Aggregator(1 << 20)
    try:
        res = agg.aggregate_batched([(k.to(DEV), [p.to(DEV) for p in pay]) for k, pay in insts], aggs,
                                    capacities=[10, 30_000, 100])
        assert res[0] is None  # 4000 rows over 4000 values need more than 10 rows
        for (k, pay), r in zip(insts[1:], res[1:]):
            ok, oa = agg.aggregate([k.to(DEV)], [p.to(DEV) for p in pay], aggs)
            np.testing.assert_array_equal(to_np(r[0]), to_np(ok[0]))
            for a in range(len(aggs)):
                np.testing.assert_array_equal(to_np(r[1][a]), to_np(oa[a]))
    finally:
        agg.close()

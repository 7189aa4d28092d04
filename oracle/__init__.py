"""CPU oracle for sort-based grouping and aggregation (arXiv 2010.00152).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2010_00152_gb300``) never imports it and shares no code with it.

The arithmetic lives in ``sgagg_oracle.c`` (plain C: normalize keys, sort the
(key, row) pairs with ``qsort``, fold equal keys in one in-stream pass).  This
module only marshals numpy arrays into it, and composes those steps for the
hybrid run generation of Sec. 5.2.3.  ``spill_model`` holds the paper's
closed-form spill analysis.

Aggregate codes follow the problem statement of Sec. 1 (count(*), sum, min,
max): COUNT=0, SUM=1, MIN=2, MAX=3.
"""
import ctypes
import numpy as np

from . import build as _build

COUNT, SUM, MIN, MAX = 0, 1, 2, 3

_lib = None


def lib():
    """Load (building first if needed) the oracle shared library."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        i32 = ctypes.c_int
        L.orc_normalize.argtypes = [i32, P, P, i64, P]
        L.orc_normalize.restype = i32
        L.orc_unpack.argtypes = [i32, P, i32, P, i64, P]
        L.orc_unpack.restype = None
        L.orc_groupby.argtypes = [P, i64, i32, P, i32, P, P, P, P]
        L.orc_groupby.restype = i64
        L.orc_fold_states.argtypes = [P, i64, i32, P, P, P, P]
        L.orc_fold_states.restype = i64
        L.orc_run_generation.argtypes = [P, i64, i64, i32, P, i32, P, P, P, P, P]
        L.orc_run_generation.restype = i64
        L.orc_absorb_runs.argtypes = [P, i64, i64, i64, i32, P, i32, P, P, P, P]
        L.orc_absorb_runs.restype = i64
        L.orc_count_distinct.argtypes = [P, P, i64, i32, P, i32, P, P, P, P, P]
        L.orc_count_distinct.restype = i64
        _lib = L
    return _lib


def _ptrs(arrs):
    a = (ctypes.c_void_p * max(1, len(arrs)))()
    for i, x in enumerate(arrs):
        a[i] = x.ctypes.data
    return a


def _agg_arrays(aggs):
    ops = np.ascontiguousarray([int(op) for op, _ in aggs], dtype=np.int32)
    cols = np.ascontiguousarray([int(c) for _, c in aggs], dtype=np.int32)
    return ops, cols


def normalize(key_cols):
    """Order-preserving normalized key of unsigned key columns (Sec. 2.4).

    ``key_cols`` is a list of uint8/16/32/64 arrays, column 0 most significant.
    """
    key_cols = [np.ascontiguousarray(c) for c in key_cols]
    n = len(key_cols[0])
    widths = np.ascontiguousarray([c.dtype.itemsize for c in key_cols], dtype=np.int32)
    for c in key_cols:
        if c.dtype.kind != "u":
            raise TypeError("key columns are unsigned integers")
    out = np.empty(n, dtype=np.uint64)
    rc = lib().orc_normalize(len(key_cols), widths.ctypes.data, _ptrs(key_cols), n,
                             out.ctypes.data)
    if rc != 0:
        raise ValueError("key columns wider than 64 bits in total")
    return out


def unpack(keys, widths, c):
    """Column ``c`` (of widths ``widths`` in bytes) out of normalized keys."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    w = np.ascontiguousarray(widths, dtype=np.int32)
    out = np.empty(len(keys), dtype={1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[int(w[c])])
    lib().orc_unpack(len(w), w.ctypes.data, c, keys.ctypes.data, len(keys), out.ctypes.data)
    return out


def groupby(keys, payload, aggs):
    """Plain GROUP BY: returns (sorted distinct keys, [agg arrays]).

    keys: uint64[n] normalized keys; payload: list of int64[n] columns;
    aggs: list of (op, col) with op in COUNT/SUM/MIN/MAX.
    """
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    payload = [np.ascontiguousarray(p, dtype=np.int64) for p in payload]
    n = len(keys)
    ops, cols = _agg_arrays(aggs)
    out_k = np.empty(max(n, 1), dtype=np.uint64)
    out_a = [np.empty(max(n, 1), dtype=np.int64) for _ in aggs]
    g = lib().orc_groupby(keys.ctypes.data, n, len(payload), _ptrs(payload), len(aggs),
                          ops.ctypes.data, cols.ctypes.data, out_k.ctypes.data, _ptrs(out_a))
    if g < 0:
        raise ValueError("bad aggregate spec or allocation failure")
    return out_k[:g].copy(), [a[:g].copy() for a in out_a]


def fold_states(keys, states, ops):
    """Fold rows that carry partial aggregates (runs) into final rows."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    states = [np.ascontiguousarray(s, dtype=np.int64) for s in states]
    n = len(keys)
    opsa = np.ascontiguousarray(ops, dtype=np.int32)
    out_k = np.empty(max(n, 1), dtype=np.uint64)
    out_a = [np.empty(max(n, 1), dtype=np.int64) for _ in ops]
    g = lib().orc_fold_states(keys.ctypes.data, n, len(ops), opsa.ctypes.data, _ptrs(states),
                              out_k.ctypes.data, _ptrs(out_a))
    if g < 0:
        raise MemoryError("oracle allocation failed")
    return out_k[:g].copy(), [a[:g].copy() for a in out_a]


def run_generation(keys, payload, aggs, M):
    """Read-sort-write run generation with early aggregation (Sec. 3, 6.1).

    Returns (run_rows list, run_keys, run_states): run b is the folded batch
    of rows [b*M, (b+1)*M).
    """
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    payload = [np.ascontiguousarray(p, dtype=np.int64) for p in payload]
    n = len(keys)
    ops, cols = _agg_arrays(aggs)
    nb = (n + M - 1) // M if n > 0 else 0
    run_rows = np.zeros(max(nb, 1), dtype=np.int64)
    rk = np.empty(max(n, 1), dtype=np.uint64)
    rs = [np.empty(max(n, 1), dtype=np.int64) for _ in aggs]
    r = lib().orc_run_generation(keys.ctypes.data, n, int(M), len(payload), _ptrs(payload),
                                 len(aggs), ops.ctypes.data, cols.ctypes.data,
                                 run_rows.ctypes.data, rk.ctypes.data, _ptrs(rs))
    if r < 0:
        raise ValueError("bad run-generation arguments")
    tot = int(run_rows[:r].sum())
    return [int(x) for x in run_rows[:r]], rk[:tot].copy(), [s[:tot].copy() for s in rs]


def absorb_runs(keys, payload, aggs, M, B):
    """Run generation with an absorbing index of at most M keys, batches of B
    rows (Sec. 3, Sec. 6.1).  Returns (run row counts, rows left in the
    index); no runs means the input was absorbed in memory."""
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    payload = [np.ascontiguousarray(p, dtype=np.int64) for p in payload]
    n = len(keys)
    ops, cols = _agg_arrays(aggs)
    run_rows = np.zeros(n + 2, dtype=np.int64)
    left = ctypes.c_int64()
    r = lib().orc_absorb_runs(keys.ctypes.data, n, int(M), int(B), len(payload), _ptrs(payload), len(aggs),
                              ops.ctypes.data, cols.ctypes.data, run_rows.ctypes.data, ctypes.byref(left))
    if r < 0:
        raise ValueError("bad absorbing run-generation arguments")
    return [int(x) for x in run_rows[:r]], int(left.value)


def hybrid_bound(keys, M, F, f):
    """Resident key range of hybrid run generation (Sec. 5.2.3): the lowest
    keys, as many distinct keys as the index's share (1 - f/F) * M of memory
    holds.  Returns the last resident key t (keys <= t stay in memory), or
    None when no key is resident."""
    resident = int((1.0 - f / F) * M) if f < F else 0
    uk = np.unique(np.asarray(keys, dtype=np.uint64))
    if resident <= 0 or len(uk) == 0:
        return None
    return int(uk[min(resident, len(uk)) - 1])


def hybrid_runs(keys, payload, aggs, M, F, f, last):
    """Hybrid run generation with early aggregation, then one wide merge
    (Sec. 5.2.3): memory fraction 1 - f/F is an index that absorbs the rows
    of the resident key range (keys <= last; none when last is None)
    without spilling; fraction f/F runs read-sort-write cycles over the
    other rows (runs of f/F * M input rows, each folded); the final merge
    folds the runs, and the resident groups precede the merged ones in key
    order.

    Returns (run row counts, rows absorbed in memory, resident distinct keys,
    (out keys, out aggs)).
    """
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    payload = [np.ascontiguousarray(p, dtype=np.int64) for p in payload]
    res = keys <= np.uint64(last) if last is not None else np.zeros(len(keys), dtype=bool)
    rk_, ra_ = groupby(keys[res], [p[res] for p in payload], aggs)
    spill = ~res
    m_run = max(1, int(f / F * M)) if f > 0 else max(1, len(keys))
    runs, sk, ss = run_generation(keys[spill], [p[spill] for p in payload], aggs, m_run)
    mk, ma = fold_states(sk, ss, [op for op, _ in aggs])
    out_k = np.concatenate([rk_, mk])
    out_a = [np.concatenate([a, b]) for a, b in zip(ra_, ma)]
    return runs, int(res.sum()), len(rk_), (out_k, out_a)


def count_distinct(key_cols, ucol, payload, aggs):
    """count(distinct u) per group of the key columns, with aggs over all
    rows of each group: (group key columns, distinct counts, agg arrays)."""
    widths = [np.asarray(c).dtype.itemsize for c in key_cols]
    g = normalize(key_cols)
    u = np.ascontiguousarray(np.asarray(ucol).astype(np.uint64))
    payload = [np.ascontiguousarray(p, dtype=np.int64) for p in payload]
    n = len(g)
    ops, cols = _agg_arrays(aggs)
    ok = np.empty(max(n, 1), dtype=np.uint64)
    od = np.empty(max(n, 1), dtype=np.int64)
    oa = [np.empty(max(n, 1), dtype=np.int64) for _ in aggs]
    r = lib().orc_count_distinct(g.ctypes.data, u.ctypes.data, n, len(payload), _ptrs(payload), len(aggs),
                                 ops.ctypes.data, cols.ctypes.data, ok.ctypes.data, od.ctypes.data, _ptrs(oa))
    if r < 0:
        raise ValueError("bad count-distinct arguments")
    return ([unpack(ok[:r], widths, c) for c in range(len(key_cols))], od[:r].copy(), [a[:r].copy() for a in oa])


def aggregate(key_cols, payload, aggs):
    """Full oracle over raw key columns: (out key columns, agg arrays)."""
    widths = [np.asarray(c).dtype.itemsize for c in key_cols]
    keys = normalize(key_cols)
    ok, oa = groupby(keys, payload, aggs)
    return [unpack(ok, widths, c) for c in range(len(key_cols))], oa

"""Python binding of the sgagg C ABI (include/sgagg.h).

Argument marshalling only: every step of the grouping path runs in the CUDA
library ``libsgagg.so``.  Function names match the C ABI; ``Aggregator`` is a
small convenience wrapper that takes torch tensors (used only for device
memory and streams) and returns torch tensors.

There is no CPU fallback: if the library is not built, or no CUDA device is
present when a call needs one, the call raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsgagg.so")

SGAGG_OK, SGAGG_EINVAL, SGAGG_ENOMEM, SGAGG_ECUDA, SGAGG_ETIMEOUT, SGAGG_ECAPACITY, SGAGG_ESTATE = range(7)
STATUS_NAMES = {0: "SGAGG_OK", 1: "SGAGG_EINVAL", 2: "SGAGG_ENOMEM", 3: "SGAGG_ECUDA",
                4: "SGAGG_ETIMEOUT", 5: "SGAGG_ECAPACITY", 6: "SGAGG_ESTATE"}
SGAGG_COUNT, SGAGG_SUM, SGAGG_MIN, SGAGG_MAX = range(4)
(SGAGG_OPT_PREFOLD, SGAGG_OPT_ARENA_CAP, SGAGG_OPT_RADIX_BITS, SGAGG_OPT_SPIN_LIMIT,
 SGAGG_OPT_FANIN_CAP, SGAGG_OPT_FAULT_ALLOC, SGAGG_OPT_TIMING, SGAGG_OPT_TEST_STALL,
 SGAGG_OPT_POLICY, SGAGG_OPT_ABSORB_BATCH, SGAGG_OPT_LOWCARD, SGAGG_OPT_MERGE_THREADS,
 SGAGG_OPT_HYBRID_FANIN, SGAGG_OPT_HYBRID_F, SGAGG_OPT_HYBRID_LAST, SGAGG_OPT_HYBRID_LAST_AUTO,
 SGAGG_OPT_MERGE_COPY, SGAGG_OPT_PREFOLD_BINS, SGAGG_OPT_PREFOLD_ROWS, SGAGG_OPT_ONE_PASS,
 SGAGG_OPT_PART_LEVELS, SGAGG_OPT_BATCH_GROUP_ROWS, SGAGG_OPT_TIMING_CLASSES) = range(23)


class sgagg_agg(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("col", ctypes.c_int32)]


class sgagg_spec(ctypes.Structure):
    _fields_ = [("n_aggs", ctypes.c_int32), ("aggs", ctypes.POINTER(sgagg_agg))]


class sgagg_keys(ctypes.Structure):
    _fields_ = [("n_cols", ctypes.c_int32), ("bytes", ctypes.POINTER(ctypes.c_int32)),
                ("cols", ctypes.POINTER(ctypes.c_void_p))]


KERNEL_CLASSES = ("probe", "hist", "plan", "scatter", "prefold", "rungen", "merge", "other", "stream")


class sgagg_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in (
        "n_rows", "batches", "runs", "run_rows", "run_bytes_device", "run_bytes_host",
        "peak_scratch_bytes", "out_rows", "out_bytes", "prefold_passes", "split_segments",
        "merge_tiles", "kernel_launches")] + [
        ("class_launches", ctypes.c_int64 * 9), ("class_bytes", ctypes.c_int64 * 9),
        ("class_ms", ctypes.c_double * 9), ("resident_rows", ctypes.c_int64), ("resident_keys", ctypes.c_int64),
        ("hybrid_f", ctypes.c_int64), ("one_pass", ctypes.c_int64)]

    def as_dict(self):
        d = {n: int(getattr(self, n)) for n, t in self._fields_ if t is ctypes.c_int64}
        d["kernels"] = {KERNEL_CLASSES[i]: dict(launches=int(self.class_launches[i]),
                                                bytes=int(self.class_bytes[i]),
                                                ms=float(self.class_ms[i])) for i in range(9)}
        return d


class sgagg_instance(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("key_bytes", ctypes.c_int32), ("n_payload", ctypes.c_int32),
                ("payload", ctypes.c_void_p), ("n", ctypes.c_int64), ("out_keys", ctypes.c_void_p),
                ("out_aggs", ctypes.c_void_p), ("out_capacity", ctypes.c_int64),
                ("out_rows", ctypes.c_void_p)]


class sgagg_server_config(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("device_budget_bytes", ctypes.c_int64),
                ("memory_budget_rows", ctypes.c_int64), ("small_rows", ctypes.c_int64),
                ("max_batch", ctypes.c_int32), ("max_batch_rows", ctypes.c_int64)]


class sgagg_request(ctypes.Structure):
    _fields_ = [("keys", ctypes.c_void_p), ("key_bytes", ctypes.c_int32), ("n_payload", ctypes.c_int32),
                ("payload", ctypes.c_void_p), ("n", ctypes.c_int64), ("out_keys", ctypes.c_void_p),
                ("out_aggs", ctypes.c_void_p), ("out_capacity", ctypes.c_int64), ("ready", ctypes.c_void_p)]


class sgagg_request_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("slot", ctypes.c_int32), ("rows", ctypes.c_int64),
                ("submit_ns", ctypes.c_int64), ("start_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
                ("batch_size", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_ if n != "pad"}


_lib = None


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libsgagg.so is not built; run __graft_entry__.build() "
                               "(the grouping path has no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        L.sgagg_create.argtypes = [i64, ctypes.POINTER(vp)]
        L.sgagg_set_option.argtypes = [vp, i32, i64]
        L.sgagg_aggregate.argtypes = [vp, ctypes.POINTER(sgagg_keys), vp, i32, i64,
                                      ctypes.POINTER(sgagg_spec), vp, vp, i64, vp]
        L.sgagg_aggregate_host.argtypes = [vp, ctypes.POINTER(sgagg_keys), vp, i32, i64,
                                           ctypes.POINTER(sgagg_spec), vp, vp, i64,
                                           ctypes.POINTER(i64), vp]
        L.sgagg_result_rows.argtypes = [vp, ctypes.POINTER(i64)]
        L.sgagg_temp_bytes.argtypes = [vp]
        L.sgagg_temp_bytes.restype = i64
        L.sgagg_stats.argtypes = [vp, ctypes.POINTER(sgagg_stats_t)]
        L.sgagg_aggregate_batched.argtypes = [vp, ctypes.POINTER(sgagg_instance), i32,
                                              ctypes.POINTER(sgagg_spec), vp]
        L.sgagg_aggregate_noalloc.argtypes = [ctypes.POINTER(sgagg_keys), vp, i32, i64,
                                              ctypes.POINTER(sgagg_spec), vp, vp, i64, vp, vp]
        L.sgagg_aggregate_noalloc.restype = i32
        L.sgagg_run_sizes.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
        L.sgagg_run_sizes.restype = i32
        L.sgagg_destroy.argtypes = [vp]
        L.sgagg_destroy.restype = None
        L.sgagg_last_error.argtypes = [vp]
        L.sgagg_last_error.restype = ctypes.c_char_p
        for f in ("sgagg_create", "sgagg_set_option", "sgagg_aggregate", "sgagg_aggregate_host",
                  "sgagg_result_rows", "sgagg_stats", "sgagg_aggregate_batched"):
            getattr(L, f).restype = i32
        L.sgagg_aggregate_distinct.argtypes = [vp, ctypes.POINTER(sgagg_keys), vp, i32, vp, i32, i64,
                                               ctypes.POINTER(sgagg_spec), vp, vp, vp, i64, vp]
        L.sgagg_aggregate_distinct.restype = i32
        dp = ctypes.POINTER(ctypes.c_double)
        L.sgagg_request_footprint.argtypes = [i64, i32, i32, i32, i64, i64]
        L.sgagg_request_footprint.restype = i64
        L.sgagg_server_now_ns.argtypes = []
        L.sgagg_server_now_ns.restype = i64
        L.sgagg_server_create.argtypes = [ctypes.POINTER(sgagg_server_config), ctypes.POINTER(sgagg_spec),
                                          ctypes.POINTER(vp)]
        L.sgagg_server_submit.argtypes = [vp, ctypes.POINTER(sgagg_request), ctypes.POINTER(i64)]
        L.sgagg_server_wait.argtypes = [vp, i64, ctypes.POINTER(sgagg_request_result)]
        L.sgagg_server_poll.argtypes = [vp, i64, ctypes.POINTER(i32), ctypes.POINTER(sgagg_request_result)]
        L.sgagg_server_destroy.argtypes = [vp]
        L.sgagg_server_destroy.restype = None
        L.sgagg_server_simulate.argtypes = [ctypes.POINTER(sgagg_server_config), i32, i32, i32,
                                            ctypes.POINTER(i64), dp, dp, dp, dp,
                                            ctypes.POINTER(i32), ctypes.POINTER(i32)]
        for f in ("sgagg_server_create", "sgagg_server_submit", "sgagg_server_wait", "sgagg_server_poll",
                  "sgagg_server_simulate"):
            getattr(L, f).restype = i32
        _lib = L
    return _lib


class SgaggError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


# ---- C ABI, same names --------------------------------------------------
def sgagg_create(memory_budget_rows):
    h = ctypes.c_void_p()
    st = lib().sgagg_create(int(memory_budget_rows), ctypes.byref(h))
    if st != SGAGG_OK:
        raise SgaggError(st, "sgagg_create(%d)" % memory_budget_rows)
    return h


def sgagg_last_error(h):
    m = lib().sgagg_last_error(h)
    return m.decode() if m else ""


def _check(h, st):
    if st != SGAGG_OK:
        raise SgaggError(st, sgagg_last_error(h))


def sgagg_set_option(h, key, value):
    _check(h, lib().sgagg_set_option(h, int(key), int(value)))


def sgagg_destroy(h):
    lib().sgagg_destroy(h)


def sgagg_temp_bytes(h):
    return int(lib().sgagg_temp_bytes(h))


def sgagg_result_rows(h):
    r = ctypes.c_int64()
    _check(h, lib().sgagg_result_rows(h, ctypes.byref(r)))
    return int(r.value)


def sgagg_stats(h):
    s = sgagg_stats_t()
    _check(h, lib().sgagg_stats(h, ctypes.byref(s)))
    return s.as_dict()


def sgagg_run_sizes(h):
    """Rows of each run the last call wrote, in the order written."""
    cnt = ctypes.c_int64()
    _check(h, lib().sgagg_run_sizes(h, None, 0, ctypes.byref(cnt)))
    buf = (ctypes.c_int64 * max(1, cnt.value))()
    _check(h, lib().sgagg_run_sizes(h, buf, cnt.value, ctypes.byref(cnt)))
    return [int(buf[i]) for i in range(cnt.value)]


class _Args:
    """Keeps ctypes argument structures alive for one call."""

    def __init__(self, key_ptrs, key_bytes, payload_ptrs, aggs, out_key_ptrs, out_agg_ptrs):
        nk = len(key_ptrs)
        self.kb = (ctypes.c_int32 * nk)(*key_bytes)
        self.kc = (ctypes.c_void_p * nk)(*key_ptrs)
        self.keys = sgagg_keys(nk, self.kb, self.kc)
        self.pay = (ctypes.c_void_p * max(1, len(payload_ptrs)))(*payload_ptrs)
        self.aggs = (sgagg_agg * max(1, len(aggs)))(*[sgagg_agg(int(o), int(c)) for o, c in aggs])
        self.spec = sgagg_spec(len(aggs), self.aggs)
        self.ok = (ctypes.c_void_p * nk)(*out_key_ptrs)
        self.oa = (ctypes.c_void_p * max(1, len(out_agg_ptrs)))(*out_agg_ptrs)


def sgagg_aggregate(h, key_ptrs, key_bytes, payload_ptrs, n, aggs, out_key_ptrs, out_agg_ptrs,
                    out_capacity, stream=0):
    """Raw call with integer device pointers."""
    a = _Args(key_ptrs, key_bytes, payload_ptrs, aggs, out_key_ptrs, out_agg_ptrs)
    st = lib().sgagg_aggregate(h, ctypes.byref(a.keys), a.pay, len(payload_ptrs), int(n),
                               ctypes.byref(a.spec), a.ok, a.oa, int(out_capacity),
                               ctypes.c_void_p(stream))
    _check(h, st)


def sgagg_aggregate_host(h, key_ptrs, key_bytes, payload_ptrs, n, aggs, out_key_ptrs, out_agg_ptrs,
                         out_capacity, stream=0):
    """Raw call with integer HOST pointers; returns the number of rows."""
    a = _Args(key_ptrs, key_bytes, payload_ptrs, aggs, out_key_ptrs, out_agg_ptrs)
    rows = ctypes.c_int64()
    st = lib().sgagg_aggregate_host(h, ctypes.byref(a.keys), a.pay, len(payload_ptrs), int(n),
                                    ctypes.byref(a.spec), a.ok, a.oa, int(out_capacity),
                                    ctypes.byref(rows), ctypes.c_void_p(stream))
    _check(h, st)
    return int(rows.value)


def sgagg_aggregate_distinct(h, key_ptrs, key_bytes, distinct_ptr, distinct_bytes, payload_ptrs, n, aggs,
                             out_key_ptrs, out_distinct_ptr, out_agg_ptrs, out_capacity, stream=0):
    """Raw call with integer device pointers: count(distinct u) per group."""
    a = _Args(key_ptrs, key_bytes, payload_ptrs, aggs, out_key_ptrs, out_agg_ptrs)
    st = lib().sgagg_aggregate_distinct(h, ctypes.byref(a.keys), ctypes.c_void_p(distinct_ptr), int(distinct_bytes),
                                        a.pay, len(payload_ptrs), int(n), ctypes.byref(a.spec), a.ok,
                                        ctypes.c_void_p(out_distinct_ptr), a.oa, int(out_capacity),
                                        ctypes.c_void_p(stream))
    _check(h, st)


NOALLOC_MAX_ROWS = 8192


def sgagg_aggregate_noalloc(key_ptrs, key_bytes, payload_ptrs, n, aggs, out_key_ptrs, out_agg_ptrs,
                            out_capacity, out_rows_ptr, stream=0):
    """Handle-free grouping of at most NOALLOC_MAX_ROWS rows that allocates no
    memory (device pointers in and out; the row count lands in the device
    int64 at out_rows_ptr, -1 if out_capacity was too small)."""
    a = _Args(key_ptrs, key_bytes, payload_ptrs, aggs, out_key_ptrs, out_agg_ptrs)
    st = lib().sgagg_aggregate_noalloc(ctypes.byref(a.keys), a.pay, len(payload_ptrs), int(n),
                                       ctypes.byref(a.spec), a.ok, a.oa, int(out_capacity),
                                       ctypes.c_void_p(out_rows_ptr), ctypes.c_void_p(stream))
    if st != SGAGG_OK:
        raise SgaggError(st, sgagg_last_error(None))


def sgagg_aggregate_batched(h, instances, aggs, stream=0):
    """instances: list of sgagg_instance (device pointers inside)."""
    arr = (sgagg_instance * max(1, len(instances)))(*instances)
    aa = (sgagg_agg * max(1, len(aggs)))(*[sgagg_agg(int(o), int(c)) for o, c in aggs])
    spec = sgagg_spec(len(aggs), aa)
    _check(h, lib().sgagg_aggregate_batched(h, arr, len(instances), ctypes.byref(spec),
                                            ctypes.c_void_p(stream)))


# ---- convenience wrapper over torch tensors ------------------------------
OPTION_NAMES = {"prefold": SGAGG_OPT_PREFOLD, "arena_cap": SGAGG_OPT_ARENA_CAP,
                "radix_bits": SGAGG_OPT_RADIX_BITS, "spin_limit": SGAGG_OPT_SPIN_LIMIT,
                "fanin_cap": SGAGG_OPT_FANIN_CAP, "fault_alloc": SGAGG_OPT_FAULT_ALLOC,
                "timing": SGAGG_OPT_TIMING, "test_stall": SGAGG_OPT_TEST_STALL,
                "policy": SGAGG_OPT_POLICY, "absorb_batch": SGAGG_OPT_ABSORB_BATCH,
                "lowcard": SGAGG_OPT_LOWCARD, "merge_threads": SGAGG_OPT_MERGE_THREADS,
                "hybrid_fanin": SGAGG_OPT_HYBRID_FANIN, "hybrid_f": SGAGG_OPT_HYBRID_F,
                "hybrid_last": SGAGG_OPT_HYBRID_LAST, "merge_copy": SGAGG_OPT_MERGE_COPY,
                "prefold_bins": SGAGG_OPT_PREFOLD_BINS, "prefold_rows": SGAGG_OPT_PREFOLD_ROWS,
                "one_pass": SGAGG_OPT_ONE_PASS, "part_levels": SGAGG_OPT_PART_LEVELS,
                "batch_group_rows": SGAGG_OPT_BATCH_GROUP_ROWS, "timing_classes": SGAGG_OPT_TIMING_CLASSES}

# The options the autotuner may set, with the library's defaults (restored
# when a later call's shape leaves one out).  All of them leave results
# unchanged.
TUNABLE_DEFAULTS = {"prefold": -1, "radix_bits": 0, "fanin_cap": 0, "merge_copy": 0, "prefold_bins": 0,
                    "prefold_rows": 8192, "one_pass": 1, "part_levels": 0, "batch_group_rows": 1 << 25,
                    "lowcard": 1, "merge_threads": 0}


class Aggregator:
    """One handle.  aggregate() groups device tensors and returns tensors.

    autotune=True: before every call, the options the autotuner's cache
    (tuning.py; `cache` = another cache file) gives for the call's shape are
    set -- the duplicate share from the handle's previous call of the same
    kind, when there was one.  Options passed here explicitly are left as
    given.  `last_autotune` tells what was chosen."""

    def __init__(self, memory_budget_rows, autotune=False, cache=None, **options):
        self.h = sgagg_create(memory_budget_rows)
        for k, v in options.items():
            self.set_option(OPTION_NAMES[k], v)
        self.autotune = autotune
        self._cache_path = cache
        self._cache = None
        self._user = set(options)
        self._tuned = {}
        self._last_dup = {}
        self.last_autotune = None

    def _apply_tuning(self, call, n_rows, key_bits, n_aggs):
        from . import tuning
        if self._cache is None:
            self._cache = tuning.load(self._cache_path or tuning.CACHE)
        key = tuning.shape_key(call, n_rows, key_bits, n_aggs, self._last_dup.get(call))
        opts, source, matched = tuning.choose(key, self._cache)
        opts = {k: v for k, v in opts.items() if k in TUNABLE_DEFAULTS and k not in self._user}
        for k in [k for k in self._tuned if k not in opts]:
            self.set_option(OPTION_NAMES[k], TUNABLE_DEFAULTS[k])
            del self._tuned[k]
        for k, v in opts.items():
            if self._tuned.get(k) != v:
                self.set_option(OPTION_NAMES[k], v)
                self._tuned[k] = v
        self.last_autotune = {"shape": key, "options": opts, "source": source, "matched": matched}

    def _record_dup(self, call):
        st = sgagg_stats(self.h)
        if st["n_rows"] > 0:
            self._last_dup[call] = 1.0 - st["out_rows"] / st["n_rows"]

    def close(self):
        if self.h is not None:
            sgagg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key, value):
        if key == SGAGG_OPT_HYBRID_LAST and value >= 1 << 63:
            value -= 1 << 64  # the key's 64 bits through the int64 argument
        sgagg_set_option(self.h, key, value)

    def aggregate(self, key_cols, payload, aggs, capacity=None, out=None, stream=None, sync=True):
        """key_cols: list of unsigned CUDA tensors (uint8/16/32/64); payload:
        list of int64 CUDA tensors; aggs: list of (op, col).  Returns
        (key column tensors, aggregate tensors) trimmed to the output rows."""
        import torch
        n = int(key_cols[0].numel()) if key_cols else 0
        cap = n if capacity is None else int(capacity)
        dev = key_cols[0].device
        if out is None:
            ok = [torch.empty(max(1, cap), dtype=k.dtype, device=dev) for k in key_cols]
            oa = [torch.empty(max(1, cap), dtype=torch.int64, device=dev) for _ in aggs]
        else:
            ok, oa = out
        s = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
        if self.autotune:
            self._apply_tuning("aggregate", n, 8 * sum(k.element_size() for k in key_cols), len(aggs))
        sgagg_aggregate(self.h, [k.data_ptr() for k in key_cols], [k.element_size() for k in key_cols],
                        [p.data_ptr() for p in payload], n, aggs, [k.data_ptr() for k in ok],
                        [a.data_ptr() for a in oa], cap, s)
        if not sync:
            return ok, oa
        rows = sgagg_result_rows(self.h)
        if self.autotune:
            self._record_dup("aggregate")
        return [k[:rows] for k in ok], [a[:rows] for a in oa]

    def aggregate_batched(self, instances, aggs, capacities=None, stream=None):
        """instances: list of (key tensor (one unsigned column), [int64 payload
        tensors]) on one CUDA device.  Groups every instance independently in
        one batched call; returns a list of (keys, [aggregates]) per instance
        (None for an instance whose capacity was too small)."""
        import torch
        dev = instances[0][0].device if instances else torch.device("cuda")
        keep = []
        descs = []
        outs = []
        rows = torch.zeros(max(1, len(instances)), dtype=torch.int64, device=dev)
        for i, (k, pay) in enumerate(instances):
            n = int(k.numel())
            cap = n if capacities is None else int(capacities[i])
            ok = torch.empty(max(1, cap), dtype=k.dtype, device=dev)
            oa = [torch.empty(max(1, cap), dtype=torch.int64, device=dev) for _ in aggs]
            pp = torch.tensor([p.data_ptr() for p in pay] or [0], dtype=torch.int64, device=dev)
            op = torch.tensor([a.data_ptr() for a in oa] or [0], dtype=torch.int64, device=dev)
            keep += [k, ok, pp, op] + list(pay) + oa
            descs.append(sgagg_instance(k.data_ptr(), k.element_size(), len(pay), pp.data_ptr(), n, ok.data_ptr(),
                                        op.data_ptr(), cap, rows.data_ptr() + 8 * i))
            outs.append((ok, oa))
        s = stream if stream is not None else torch.cuda.current_stream(dev).cuda_stream
        if self.autotune:
            self._apply_tuning("batched", sum(int(k.numel()) for k, _ in instances),
                               8 * max([k.element_size() for k, _ in instances] or [1]), len(aggs))
        sgagg_aggregate_batched(self.h, descs, aggs, s)
        torch.cuda.synchronize(dev)
        if self.autotune:
            self._record_dup("batched")
        r = rows.cpu().tolist()
        res = []
        for i, (ok, oa) in enumerate(outs):
            res.append(None if r[i] < 0 else (ok[:r[i]], [a[:r[i]] for a in oa]))
        del keep
        return res

    def rows(self):
        return sgagg_result_rows(self.h)

    def stats(self):
        return sgagg_stats(self.h)

    def run_sizes(self):
        return sgagg_run_sizes(self.h)

    def temp_bytes(self):
        return sgagg_temp_bytes(self.h)

    def aggregate_distinct(self, key_cols, ucol, payload, aggs, capacity=None):
        """count(distinct ucol) per group of key_cols, with aggs over all rows
        of each group.  Returns (group key columns, distinct counts, aggs)."""
        import torch
        n = int(key_cols[0].numel()) if key_cols else 0
        cap = n if capacity is None else int(capacity)
        dev = key_cols[0].device
        ok = [torch.empty(max(1, cap), dtype=k.dtype, device=dev) for k in key_cols]
        od = torch.empty(max(1, cap), dtype=torch.int64, device=dev)
        oa = [torch.empty(max(1, cap), dtype=torch.int64, device=dev) for _ in aggs]
        s = torch.cuda.current_stream(dev).cuda_stream
        sgagg_aggregate_distinct(self.h, [k.data_ptr() for k in key_cols], [k.element_size() for k in key_cols],
                                 ucol.data_ptr(), ucol.element_size(), [p.data_ptr() for p in payload], n, aggs,
                                 [k.data_ptr() for k in ok], od.data_ptr(), [a.data_ptr() for a in oa], cap, s)
        rows = sgagg_result_rows(self.h)
        return [k[:rows] for k in ok], od[:rows], [a[:rows] for a in oa]

    def aggregate_host(self, key_cols, payload, aggs, capacity=None, stream=0):
        """Host numpy arrays in, host numpy arrays out (copies inside the call)."""
        import numpy as np
        n = len(key_cols[0])
        cap = n if capacity is None else int(capacity)
        key_cols = [np.ascontiguousarray(k) for k in key_cols]
        payload = [np.ascontiguousarray(p, dtype=np.int64) for p in payload]
        ok = [np.empty(max(1, cap), dtype=k.dtype) for k in key_cols]
        oa = [np.empty(max(1, cap), dtype=np.int64) for _ in aggs]
        rows = sgagg_aggregate_host(self.h, [k.ctypes.data for k in key_cols],
                                    [k.dtype.itemsize for k in key_cols],
                                    [p.ctypes.data for p in payload], n, aggs,
                                    [k.ctypes.data for k in ok], [a.ctypes.data for a in oa], cap,
                                    stream)
        return [k[:rows] for k in ok], [a[:rows] for a in oa]


# ---- serving --------------------------------------------------------------
def server_config(slots=8, device_budget_bytes=64 << 30, memory_budget_rows=1 << 22, small_rows=1 << 16,
                  max_batch=256, max_batch_rows=1 << 24):
    return sgagg_server_config(int(slots), int(device_budget_bytes), int(memory_budget_rows), int(small_rows),
                               int(max_batch), int(max_batch_rows))


def sgagg_request_footprint(n, key_bytes, n_payload, n_aggs, out_capacity, memory_budget_rows):
    return int(lib().sgagg_request_footprint(int(n), int(key_bytes), int(n_payload), int(n_aggs),
                                             int(out_capacity), int(memory_budget_rows)))


def sgagg_server_now_ns():
    return int(lib().sgagg_server_now_ns())


def sgagg_server_simulate(cfg, n_payload, n_aggs, rows, arrive_us, cost_us):
    """Run the server's admission and batching decisions on the host against
    a cost model; returns (start_us, finish_us, slot, batch) lists."""
    n = len(rows)
    r = (ctypes.c_int64 * max(1, n))(*[int(x) for x in rows])
    a = (ctypes.c_double * max(1, n))(*[float(x) for x in arrive_us])
    c = (ctypes.c_double * 3)(*[float(x) for x in cost_us])
    st_ = (ctypes.c_double * max(1, n))()
    fi = (ctypes.c_double * max(1, n))()
    sl = (ctypes.c_int32 * max(1, n))()
    bt = (ctypes.c_int32 * max(1, n))()
    s = lib().sgagg_server_simulate(ctypes.byref(cfg), int(n_payload), int(n_aggs), n, r, a, c, st_, fi, sl, bt)
    if s != SGAGG_OK:
        raise SgaggError(s, "sgagg_server_simulate")
    return list(st_)[:n], list(fi)[:n], list(sl)[:n], list(bt)[:n]


class Server:
    """Request loop (sgagg_server_*) over torch tensors: submit() queues a
    request and returns a ticket; wait()/poll() give its result dict and its
    output tensors.  Tensors of a request are kept alive until it is done."""

    def __init__(self, aggs, **cfg):
        self.aggs = list(aggs)
        self.cfg = server_config(**cfg)
        self._aggs = (sgagg_agg * max(1, len(self.aggs)))(*[sgagg_agg(int(o), int(c)) for o, c in self.aggs])
        self._spec = sgagg_spec(len(self.aggs), self._aggs)
        self.h = ctypes.c_void_p()
        st = lib().sgagg_server_create(ctypes.byref(self.cfg), ctypes.byref(self._spec), ctypes.byref(self.h))
        if st != SGAGG_OK:
            raise SgaggError(st, "sgagg_server_create")
        self._live = {}

    def submit(self, keys, payload, capacity=None, ready=None, out=None):
        import torch
        n = keys.numel()
        cap = n if capacity is None else int(capacity)
        if out is None:
            ok = torch.empty(max(1, cap), dtype=keys.dtype, device=keys.device)
            oa = [torch.empty(max(1, cap), dtype=torch.int64, device=keys.device) for _ in self.aggs]
        else:
            ok, oa = out
        pay = (ctypes.c_void_p * max(1, len(payload)))(*[p.data_ptr() for p in payload])
        oap = (ctypes.c_void_p * max(1, len(oa)))(*[a.data_ptr() for a in oa])
        req = sgagg_request(keys.data_ptr(), keys.element_size(), len(payload), ctypes.cast(pay, ctypes.c_void_p),
                            n, ok.data_ptr(), ctypes.cast(oap, ctypes.c_void_p), cap,
                            ready.cuda_event if ready is not None else None)
        t = ctypes.c_int64()
        st = lib().sgagg_server_submit(self.h, ctypes.byref(req), ctypes.byref(t))
        if st != SGAGG_OK:
            raise SgaggError(st, "sgagg_server_submit")
        self._live[t.value] = (keys, payload, ok, oa, ready)
        return t.value

    def _finish(self, t, r):
        keys, payload, ok, oa, ready = self._live.pop(t)
        d = r.as_dict()
        rows = d["rows"]
        d["out"] = (ok[:rows], [a[:rows] for a in oa]) if rows >= 0 else None
        return d

    def wait(self, t):
        r = sgagg_request_result()
        st = lib().sgagg_server_wait(self.h, int(t), ctypes.byref(r))
        if st != SGAGG_OK:
            raise SgaggError(st, "sgagg_server_wait")
        return self._finish(t, r)

    def poll(self, t):
        r = sgagg_request_result()
        done = ctypes.c_int32()
        st = lib().sgagg_server_poll(self.h, int(t), ctypes.byref(done), ctypes.byref(r))
        if st != SGAGG_OK:
            raise SgaggError(st, "sgagg_server_poll")
        return self._finish(t, r) if done.value else None

    def close(self):
        if self.h:
            lib().sgagg_server_destroy(self.h)
            self.h = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

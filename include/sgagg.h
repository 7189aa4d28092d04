/*
 * sgagg.h -- C ABI of a GPU (sm_103a) implementation of sort-based grouping
 * and aggregation with early aggregation during run generation and wide
 * merging (Do, Graefe, Naughton, "Efficient sorting, duplicate removal,
 * grouping, and aggregation", arXiv 2010.00152).
 *
 * Operation (Sec. 1, "select A, B, count(*), sum(X), min(Z), max(Y) ...
 * group by A, B"; Sec. 3.3 on intermediate rows carrying partial aggregates;
 * Sec. 6.1 on sorted output): one output row per distinct key, keys strictly
 * ascending (unsigned, lexicographic over the key columns), with int64
 * count(*), sum (wrapping modulo 2^64), min and max (signed) per requested
 * aggregate.  The result is unique and bit-exact.
 *
 * Method (Sec. 3, Sec. 4, Sec. 6.1):
 *   - the input is consumed in batches of memory_budget_rows rows
 *     (read-sort-write cycles); each batch is sorted and its equal keys folded
 *     before its run is written (early aggregation), so a run holds each key
 *     of its batch once;
 *   - one wide merge consumes all runs at once, folding equal keys across
 *     runs, and emits the final sorted output; a batch that covers the whole
 *     input is written straight to the output (no run, no merge).
 *
 * Conventions for every call:
 *   - Pointers named "device" must point to memory the current CUDA device
 *     can access (device memory, or mapped/managed memory).  Arrays *of*
 *     pointers (key columns, payload columns, output columns) are host arrays
 *     that the call reads before it returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is stream-ordered.  sgagg_aggregate may synchronize the
 *     stream internally while planning (it reads small counters back); all
 *     results are final once sgagg_result_rows returns SGAGG_OK.
 *   - The caller owns every input and output buffer; the library never frees
 *     them and never writes to inputs.  The handle owns its workspace, run
 *     arena and pinned host buffers; sgagg_destroy frees them.
 *   - A handle is one logical sequence of calls and is not thread-safe.  Use
 *     one handle per host thread.
 *   - Errors are status codes; sgagg_last_error(h) gives a message.  Argument
 *     errors are reported before any GPU work is enqueued.
 */
#ifndef SGAGG_H
#define SGAGG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sgagg_ctx *sgagg_t;

typedef enum {
    SGAGG_OK = 0,
    SGAGG_EINVAL = 1,    /* bad argument (null pointer, n < 0, bad spec, key wider than 64 bits) */
    SGAGG_ENOMEM = 2,    /* device or pinned host allocation failed */
    SGAGG_ECUDA = 3,     /* a CUDA runtime call failed */
    SGAGG_ETIMEOUT = 4,  /* a bounded device-side wait gave up (see SGAGG_OPT_SPIN_LIMIT) */
    SGAGG_ECAPACITY = 5, /* out_capacity smaller than the number of distinct keys */
    SGAGG_ESTATE = 6     /* call out of order (e.g. result_rows before any aggregate) */
} sgagg_status;

/* Aggregates of the problem statement (Sec. 1): count(*), sum, min, max. */
typedef enum { SGAGG_COUNT = 0, SGAGG_SUM = 1, SGAGG_MIN = 2, SGAGG_MAX = 3 } sgagg_op;

/* One aggregate: op over payload column `col` (ignored for COUNT). */
typedef struct {
    int32_t op;
    int32_t col;
} sgagg_agg;

/* The aggregate list; output column a holds aggregate a. */
typedef struct {
    int32_t n_aggs;          /* 0 .. 32; 0 = duplicate removal (keys only) */
    const sgagg_agg *aggs;   /* host array of n_aggs entries */
} sgagg_spec;

/*
 * Key columns, column 0 most significant.  Each column is an unsigned
 * integer array of 1, 2, 4 or 8 bytes per row; the widths add up to at most
 * 8 bytes.  They are combined into one order-preserving normalized key
 * (Sec. 2.4, normalized keys), so the output order is the lexicographic
 * order of the key tuples.
 */
typedef struct {
    int32_t n_cols;              /* 1 .. 8 */
    const int32_t *bytes;        /* host array: width of each column in bytes */
    const void *const *cols;     /* host array of device pointers, one per column */
} sgagg_keys;

/* Counters of the last call on the handle (any grouping entry point). */
typedef struct {
    int64_t n_rows;              /* input rows */
    int64_t batches;             /* ceil(n / memory_budget_rows) */
    int64_t runs;                /* runs written (0 when one batch covers the input) */
    int64_t run_rows;            /* rows written to all runs (the paper's spill volume) */
    int64_t run_bytes_device;    /* bytes of runs held in the device arena */
    int64_t run_bytes_host;      /* bytes of runs spilled to pinned host memory */
    int64_t peak_scratch_bytes;  /* workspace bytes in use (sort buffers, tables, status) */
    int64_t out_rows;            /* distinct keys */
    int64_t out_bytes;           /* output bytes (key columns + aggregates) */
    int64_t prefold_passes;      /* tile-level pre-aggregation passes run */
    int64_t split_segments;      /* key ranges that needed a recursive split */
    int64_t merge_tiles;         /* tiles of the wide merge */
    int64_t kernel_launches;     /* kernels launched by the call */
    /* Per kernel class (see SGAGG_K_*): launches, compulsory bytes (every
     * input of the launch read once, every output written once) and, with
     * SGAGG_OPT_TIMING, the summed CUDA-event time of the launches in ms. */
    int64_t class_launches[9];
    int64_t class_bytes[9];
    double class_ms[9];
    /* SGAGG_OPT_POLICY 2 (hybrid run generation): rows absorbed by the
     * in-memory index, its distinct keys, and the fan-out f used. */
    int64_t resident_rows;
    int64_t resident_keys;
    int64_t hybrid_f;
    /* 1 when the runs of all batches were generated in one pass per step
     * (small batches, SGAGG_OPT_ONE_PASS), else 0. */
    int64_t one_pass;
} sgagg_stats_t;

/* Kernel classes of sgagg_stats_t. */
enum {
    SGAGG_K_PROBE = 0,      /* key sample / key range */
    SGAGG_K_HIST = 1,       /* per-tile digit histogram */
    SGAGG_K_PLAN = 2,       /* tile scans and chunk planner */
    SGAGG_K_SCATTER = 3,    /* rows to their key-range bucket */
    SGAGG_K_PREFOLD = 4,    /* tile sort+fold before partitioning */
    SGAGG_K_RUNGEN = 5,     /* chunk sort+fold writing a run (or the output) */
    SGAGG_K_MERGE = 6,      /* wide merge: sort+fold of merge tiles */
    SGAGG_K_OTHER = 7,      /* copies: gathers of split key ranges, the batched call's
                               output copy, the absorbing index's runs, the
                               count(distinct) regroup */
    SGAGG_K_STREAM = 8      /* one streaming fold of a batch whose keys take few values
                               (at most 16 distinct keys in the planner's sample) */
};

/* Options for sgagg_set_option. */
typedef enum {
    SGAGG_OPT_PREFOLD = 0,        /* -1 auto (sampled duplicate rate), 0 off, 1 on */
    SGAGG_OPT_ARENA_CAP = 1,      /* max bytes of runs kept in device memory; more spill
                                     to pinned host memory.  Default: no cap (-1). */
    SGAGG_OPT_RADIX_BITS = 2,     /* bits of the batch partitioning digit, 0 = auto (1..15) */
    SGAGG_OPT_SPIN_LIMIT = 3,     /* iteration cap of device-side waits (default 1<<26);
                                     exceeded -> SGAGG_ETIMEOUT, no hang */
    SGAGG_OPT_FANIN_CAP = 4,      /* max runs in one wide merge; more runs get preliminary
                                     merges of the smallest runs first (Sec. 4.3). 0 = auto */
    SGAGG_OPT_FAULT_ALLOC = 5,    /* test hook: fail the k-th internal allocation (0 = off) */
    SGAGG_OPT_TIMING = 6,         /* 1: time every kernel class with CUDA events (class_ms) */
    SGAGG_OPT_TEST_STALL = 7,     /* test hook: 1 -- in the next sort+fold or merge launch
                                     the first chunk never publishes its row count, so the
                                     bounded waits of the others run out -> SGAGG_ETIMEOUT
                                     (no hang); 2 -- the same in the next merge launch */
    SGAGG_OPT_POLICY = 8,         /* run generation (2: hybrid, below): 0 (default) one run per batch of
                                     memory_budget_rows rows, holding the batch's distinct
                                     keys; 1 an absorbing index of at most memory_budget_rows
                                     distinct keys (Sec. 3, Sec. 6.1): each batch is sorted
                                     and folded, its distinct keys are absorbed by the index
                                     or inserted in ascending order, and when the index is
                                     full it is written as a run and emptied -- no run at all
                                     when the output fits memory_budget_rows */
    SGAGG_OPT_ABSORB_BATCH = 9,   /* rows per batch of policy 1 (0 = min(memory_budget_rows,
                                     2^22)); the runs depend on it, the result does not */
    SGAGG_OPT_LOWCARD = 10,       /* one batch whose key sample holds at most 16 distinct
                                     keys is grouped by one streaming fold (SGAGG_K_STREAM)
                                     unless this is 0; -1 (default) auto.  Same result. */
    SGAGG_OPT_MERGE_THREADS = 11, /* worker threads of one wide-merge CTA (a tile of 2048
                                     rows): 0 (default) or 256 */
    SGAGG_OPT_HYBRID_FANIN = 12,  /* policy 2: the maximal fan-in F (default 10) */
    SGAGG_OPT_HYBRID_F = 13,      /* policy 2: the actual fan-out f, 0..F; -1 (default):
                                     ceil((O - M) / (M - 1)) from the output size O
                                     estimated on the key sample, at most F */
    SGAGG_OPT_HYBRID_LAST = 14,   /* policy 2: the last key of the resident range (the
                                     normalized key's 64 bits); keys at or below it stay in
                                     the in-memory index.  Default: estimated on the key
                                     sample so that the range holds (1 - f/F) M keys */
    SGAGG_OPT_HYBRID_LAST_AUTO = 15, /* policy 2: back to the estimated resident range */
    SGAGG_OPT_MERGE_COPY = 16,    /* how the wide merge stages run slices in shared memory:
                                     0 (default) one bulk copy per slice and column
                                     (cp.async.bulk), issued by all worker warps; 1 16-byte
                                     cp.async copies by every worker thread; 2 the bulk copies
                                     issued by the control warp alone.  Same result. */
    SGAGG_OPT_PREFOLD_BINS = 17,  /* tile pre-aggregation (before runs of partial rows are
                                     sorted): 0 (default) bins a tile's rows by key range, 1 by
                                     a hash of the key.  Equal keys are adjacent either way;
                                     hashing keeps keys crowded at one end of their range
                                     (e.g. Zipf ranks used as keys) from filling a few bins.
                                     Same result. */
    SGAGG_OPT_PREFOLD_ROWS = 18,  /* rows per pre-aggregation tile of sgagg_aggregate_batched,
                                     1024..8192 (default 8192).  Same result. */
    SGAGG_OPT_ONE_PASS = 19,      /* 1 (default): when the input is several batches of more
                                     than one chunk each, at most 2^24 rows in all and few
                                     buckets, the runs of all batches are generated in one
                                     pass per step (one histogram, plan, scatter and
                                     sort+fold launch for all of them) instead of one batch
                                     at a time; 0: always a batch at a time.  The runs are
                                     the same. */
    SGAGG_OPT_PART_LEVELS = 20,   /* partitioning of a batch before its chunk sorts: 0
                                     (default) two staged levels above 2^7 buckets, else
                                     one; 1 always one level (every row written once to
                                     its final bucket).  Same result. */
    SGAGG_OPT_BATCH_GROUP_ROWS = 21, /* sgagg_aggregate_batched: rows of the multi-chunk
                                     instances grouped in one pass (2^16..2^31, default
                                     2^25); bigger groups mean fewer passes and host round
                                     trips and more scratch memory.  Same result. */
    SGAGG_OPT_TIMING_CLASSES = 22 /* with SGAGG_OPT_TIMING on: the kernel classes timed, a
                                     mask of bits 1 << SGAGG_K_* (default: all).  Two
                                     events per timed launch cost about 1.4 us of GPU time
                                     each; timing one class keeps that off the others. */
} sgagg_option;

/*
 * Create a handle.  memory_budget_rows (M >= 1) is the paper's memory size in
 * rows (Sec. 3: read-sort-write cycles make runs of memory size): with the
 * default policy the number of input rows in one batch of run generation,
 * with SGAGG_OPT_POLICY 1 the most distinct keys the absorbing index holds.
 * Returns SGAGG_EINVAL for M < 1 or out == NULL.
 */
sgagg_status sgagg_create(int64_t memory_budget_rows, sgagg_t *out);

/* Set an option (see sgagg_option).  SGAGG_EINVAL on an unknown key/value. */
sgagg_status sgagg_set_option(sgagg_t h, int32_t key, int64_t value);

/*
 * Group n input rows (device pointers) and write the sorted, aggregated
 * result.
 *   keys          key columns (device pointers), n rows each
 *   payload_cols  host array of n_payload device pointers to int64[n]
 *   spec          aggregates; SUM/MIN/MAX name a payload column
 *   out_keys      host array of keys->n_cols device pointers; column c receives
 *                 the distinct keys' column c (same width as the input column)
 *   out_aggs      host array of spec->n_aggs device pointers to int64
 *   out_capacity  rows available in every output column; n always suffices.
 *                 Fewer rows than distinct keys -> SGAGG_ECAPACITY from
 *                 sgagg_result_rows (nothing beyond out_capacity is written).
 * n == 0 is valid and yields 0 rows.  Inputs must not overlap outputs.
 */
sgagg_status sgagg_aggregate(sgagg_t h, const sgagg_keys *keys,
                             const int64_t *const *payload_cols, int32_t n_payload,
                             int64_t n, const sgagg_spec *spec,
                             void *const *out_keys, int64_t *const *out_aggs,
                             int64_t out_capacity, void *stream);

/*
 * Same operation with HOST buffers.  The inputs are copied to the device on
 * a second stream batch by batch (memory_budget_rows rows), batch b + 1
 * while batch b is grouped; the planner's key sample is read from the host
 * columns, so no copy has to finish first.  When runs are merged, the final
 * merge runs in 8 parts and each part's output is copied back while the
 * later parts merge; otherwise (one batch, or SGAGG_OPT_POLICY 1) the input
 * is copied first and the output after.  Synchronous.  *rows receives the
 * number of distinct keys.  Host buffers may be pageable; only pinned
 * buffers let the copies overlap the kernels.
 */
sgagg_status sgagg_aggregate_host(sgagg_t h, const sgagg_keys *keys,
                                  const int64_t *const *payload_cols, int32_t n_payload,
                                  int64_t n, const sgagg_spec *spec,
                                  void *const *out_keys, int64_t *const *out_aggs,
                                  int64_t out_capacity, int64_t *rows, void *stream);

/*
 * count(distinct u) per group (Sec. 7: duplicate removal followed by
 * grouping; Hypothesis 6: one sort serves both).  One grouping on the
 * composite key (group columns, u) removes duplicate (g, u) pairs -- its
 * sorted output is an interesting ordering for g -- and one in-stream pass
 * over it regroups on g without sorting again.  Output per distinct g, in
 * ascending order: the group key columns (out_keys, as in sgagg_aggregate),
 * out_distinct[i] = the number of distinct u (device int64), and every
 * aggregate of `spec` over all rows of the group.  u is one unsigned column
 * of distinct_bytes (1, 2, 4 or 8) bytes; group columns plus u must fit 8
 * bytes (SGAGG_EINVAL otherwise).  The memory budget and policy of the
 * handle apply to the first grouping.  sgagg_result_rows gives the number
 * of groups.
 */
sgagg_status sgagg_aggregate_distinct(sgagg_t h, const sgagg_keys *keys, const void *distinct_col,
                                      int32_t distinct_bytes, const int64_t *const *payload_cols,
                                      int32_t n_payload, int64_t n, const sgagg_spec *spec,
                                      void *const *out_keys, int64_t *out_distinct,
                                      int64_t *const *out_aggs, int64_t out_capacity, void *stream);

/* Synchronize the stream of the last call and return its number of output
 * rows (distinct keys), or the device-side error of that call. */
sgagg_status sgagg_result_rows(sgagg_t h, int64_t *rows);

/* Temporary bytes of the last call: bytes of all runs (device and host) plus
 * the peak workspace in use.  -1 for a NULL handle. */
int64_t sgagg_temp_bytes(sgagg_t h);

/* Counters of the last call (synchronizes its stream). */
sgagg_status sgagg_stats(sgagg_t h, sgagg_stats_t *out);

/*
 * One independent group-by instance of a batched call.  All pointers are
 * device pointers; the key is one unsigned column of key_bytes (1/2/4/8)
 * bytes per row.  *out_rows (device int64) receives the instance's distinct
 * key count, or -1 if out_capacity was too small.
 */
typedef struct {
    const void *keys;
    int32_t key_bytes;
    int32_t n_payload;
    const int64_t *const *payload;   /* device array of n_payload device pointers */
    int64_t n;
    void *out_keys;                  /* key_bytes per row */
    int64_t *const *out_aggs;        /* device array of spec->n_aggs device pointers */
    int64_t out_capacity;
    int64_t *out_rows;               /* device */
} sgagg_instance;

/*
 * Run `count` independent instances sharing one aggregate spec as one
 * grouping.  Instances of at most 8192 rows (one chunk) run in one launch,
 * a CTA each, sorted, folded and written straight to their own outputs,
 * whatever their key width.  The bigger ones are grouped together over a
 * composite normalized key (instance id above the key bits; Sec. 2.4 on
 * normalized keys): one launch pre-aggregates
 * instance-aligned tiles of every instance, the partial rows are grouped by
 * the ordinary path with partition buckets given to each instance in
 * proportion to its rows over its own key range, and one launch copies each
 * instance's rows (contiguous in the sorted output) to its outputs.  The
 * launch count does not depend on `count`: instances are taken in groups of
 * consecutive instances of up to 2^25 rows, about a dozen launches per
 * group.  When the widest key of the bigger instances plus ceil(log2(count))
 * bits exceeds 64, they run one by one through sgagg_aggregate instead.
 *
 * `inst` is a host array; the memory budget of the handle does not apply
 * (each instance is one batch, no runs).  The call synchronizes the stream
 * between groups; results are final when sgagg_result_rows returns, which
 * gives the total of all instances' rows.  An instance whose distinct keys
 * exceed its out_capacity gets *out_rows = -1 and nothing written; the
 * others are unaffected.
 */
sgagg_status sgagg_aggregate_batched(sgagg_t h, const sgagg_instance *inst, int32_t count,
                                     const sgagg_spec *spec, void *stream);

/*
 * Hybrid run generation (SGAGG_OPT_POLICY 2, Sec. 5.2.3): memory fraction
 * 1 - f/F of the budget M is an in-memory index that absorbs the rows of the
 * lowest keys -- the resident range, (1 - f/F) M distinct keys -- without
 * spilling; the other rows are grouped in read-sort-write runs of f/F * M
 * rows each, and one wide merge folds the runs.  The output is the same as
 * with any other policy.  f = 0: everything resident, no run; f = F: no
 * index, runs of M rows.  sgagg_stats gives the resident rows and keys.
 */

/*
 * Rows of each run the last call wrote (the paper's spill volume, run by run),
 * in the order written: run generation's runs, then those of preliminary
 * merges.  Copies min(*count, max_runs) entries to rows (host memory) and sets
 * *count to the number of runs.  Synchronizes with the last call's stream.
 * SGAGG_EINVAL for a null handle or count, or rows null with max_runs > 0.
 */
sgagg_status sgagg_run_sizes(sgagg_t h, int64_t *rows, int64_t max_runs, int64_t *count);

/*
 * Group at most SGAGG_NOALLOC_MAX_ROWS rows without allocating any memory.
 * The paper has no counterpart; this exists for callers that cannot allocate
 * device memory at all, e.g. code running inside a memory pool or allocator
 * callback, or a process whose allocations are reserved by a framework up
 * front: this call makes no cudaMalloc/cudaFree and no allocating library
 * call, and needs no handle.
 *
 * Same arguments as sgagg_aggregate except that there is no handle and
 * out_rows is a DEVICE pointer to one int64 that receives the number of
 * output rows, or -1 when out_capacity was too small (nothing past
 * out_capacity is written).  Asynchronous on `stream`.
 *
 * Scratch: a fixed 256-byte array in the library's device memory
 * (SGAGG_NOALLOC_SCRATCH_BYTES), held by every GPU that loads the library
 * until the process exits.  Every call shares it and overwrites it, so calls
 * whose work overlaps on the GPU (other streams, other host threads) race:
 * serialize them.  The first call on a device does a one-time set-up with
 * that device current: it looks up the array's device address
 * (cudaGetSymbolAddress) and loads every kernel this call launches (with
 * lazy module loading a kernel's first launch may load its module, which
 * allocates).  Make that first call before any stream capture and outside
 * the code that cannot allocate; every later call allocates nothing.
 *
 * Errors: n > SGAGG_NOALLOC_MAX_ROWS, or any argument error of
 * sgagg_aggregate, returns SGAGG_EINVAL before any GPU work;
 * sgagg_last_error(NULL) then gives the message.
 */
#define SGAGG_NOALLOC_MAX_ROWS 8192
#define SGAGG_NOALLOC_SCRATCH_BYTES 256
sgagg_status sgagg_aggregate_noalloc(const sgagg_keys *keys, const int64_t *const *payload_cols,
                                     int32_t n_payload, int64_t n, const sgagg_spec *spec,
                                     void *const *out_keys, int64_t *const *out_aggs,
                                     int64_t out_capacity, int64_t *out_rows, void *stream);

/*
 * Serving: a request loop over a pool of handles ("slots", one CUDA stream
 * and one host worker thread each).  The paper has no counterpart; this is
 * the system pattern built on the calls above.
 *
 *   - Requests are admitted in arrival (submit) order, never overtaking:
 *     the oldest waiting request starts as soon as a slot is free and its
 *     footprint fits what is left of device_budget_bytes.
 *   - Footprint of a request (sgagg_request_footprint): its input and
 *     output bytes plus a bound on the workspace and runs the path allocates
 *     for it.  A request whose footprint alone exceeds the budget is refused
 *     at submit with SGAGG_ECAPACITY, never queued.
 *   - Continuous batching: a request is batchable when it has at most
 *     small_rows rows and the batched call takes it in one pass (at most 8192
 *     rows, or keys of at most 4 bytes).  When the oldest waiting request is
 *     batchable, it and the batchable requests queued right behind it (up to
 *     max_batch requests and max_batch_rows rows, within the budget) run as
 *     one sgagg_aggregate_batched call.  Requests that arrive while others
 *     are on the GPU join the next batch; batches and large requests on
 *     different slots overlap on the device.
 *   - A large request runs alone through sgagg_aggregate on its slot.
 *   - slots = 1 with small_rows = 0 is the plain form: one query per call,
 *     one after another.
 *
 * Every request uses the server's aggregate spec and memory budget.  The
 * caller owns the request's device buffers and must keep them alive until
 * sgagg_server_wait (or a poll that reports it done) returns for it.
 */
typedef struct sgagg_server *sgagg_server_t;

typedef struct {
    int32_t slots;                /* >= 1 */
    int64_t device_budget_bytes;  /* admission budget over all requests in flight */
    int64_t memory_budget_rows;   /* M of every request (sgagg_create) */
    int64_t small_rows;           /* batch requests of at most this many rows; 0 = never */
    int32_t max_batch;            /* most requests in one batched call (>= 1) */
    int64_t max_batch_rows;       /* most rows in one batched call */
} sgagg_server_config;

typedef struct {
    const void *keys;               /* device, key_bytes per row */
    int32_t key_bytes;              /* 1, 2, 4 or 8 */
    int32_t n_payload;
    const int64_t *const *payload;  /* host array of n_payload device pointers */
    int64_t n;
    void *out_keys;                 /* device, out_capacity rows */
    int64_t *const *out_aggs;       /* host array of n_aggs device pointers */
    int64_t out_capacity;
    void *ready;                    /* cudaEvent_t or NULL: inputs are complete when it
                                       has fired (the slot's stream waits for it) */
} sgagg_request;

typedef struct {
    int32_t status;       /* sgagg_status of the request */
    int32_t slot;         /* slot that ran it (-1: refused) */
    int64_t rows;         /* distinct keys (-1 when status != SGAGG_OK) */
    int64_t submit_ns;    /* sgagg_server_now_ns() at submit */
    int64_t start_ns;     /* at admission */
    int64_t done_ns;      /* when its results were final */
    int32_t batch_size;   /* requests in the call that ran it (1 = alone) */
    int32_t pad;
} sgagg_request_result;

/* Footprint of a request as charged by admission, in bytes: input + output
 * bytes + 8 * m * (3 + 3C + 3(1 + S)) (workspace of one batch of
 * m = min(n, M) rows, C = payload columns, S = aggregates) + 8 * n * (1 + S)
 * when n > M (the runs) + 64 MiB. */
int64_t sgagg_request_footprint(int64_t n, int32_t key_bytes, int32_t n_payload, int32_t n_aggs,
                                int64_t out_capacity, int64_t memory_budget_rows);

/* The server's clock (monotonic, nanoseconds). */
int64_t sgagg_server_now_ns(void);

/* Start a server: cfg->slots handles and streams on the current device, one
 * worker thread each.  `spec` is copied. */
sgagg_status sgagg_server_create(const sgagg_server_config *cfg, const sgagg_spec *spec,
                                 sgagg_server_t *out);

/* Queue a request; *ticket identifies it.  Arrays of pointers in `req` are
 * copied before the call returns.  Refused (SGAGG_ECAPACITY) when its
 * footprint exceeds the budget; SGAGG_EINVAL on bad arguments. */
sgagg_status sgagg_server_submit(sgagg_server_t s, const sgagg_request *req, int64_t *ticket);

/* Block until the request is done; fill *out.  Each ticket can be waited
 * for (or polled to completion) once. */
sgagg_status sgagg_server_wait(sgagg_server_t s, int64_t ticket, sgagg_request_result *out);

/* Non-blocking: *done = 1 and *out filled when the request is done. */
sgagg_status sgagg_server_poll(sgagg_server_t s, int64_t ticket, int32_t *done, sgagg_request_result *out);

/* Finish every queued request, stop the workers, free the slots. */
void sgagg_server_destroy(sgagg_server_t s);

/*
 * The admission and batching decisions of the server, run on the host
 * against a cost model instead of the GPU (virtual time): request i of
 * rows[i] rows and 8-byte keys (footprint from sgagg_request_footprint with key_bytes 8,
 * n_payload payload columns, n_aggs aggregates and out_capacity rows[i])
 * arrives at arrive_us[i]; a call of r rows over b requests takes
 * cost_us[0] + cost_us[1] * r + cost_us[2] * b microseconds.  Writes, per
 * request, its start and finish time (us), slot, and batch id (requests
 * run by one call share it; -1 when refused).  For tests of the scheduler
 * without a GPU.
 */
sgagg_status sgagg_server_simulate(const sgagg_server_config *cfg, int32_t n_payload, int32_t n_aggs,
                                   int32_t count, const int64_t *rows, const double *arrive_us,
                                   const double *cost_us, double *start_us, double *finish_us,
                                   int32_t *slot, int32_t *batch);

/* Free the handle and everything it owns.  NULL is ignored. */
void sgagg_destroy(sgagg_t h);

/* Message of the last error on this handle ("" if none).  Valid until the
 * next call on the handle.  With h == NULL: the last message of
 * sgagg_aggregate_noalloc on this host thread. */
const char *sgagg_last_error(sgagg_t h);

#ifdef __cplusplus
}
#endif
#endif /* SGAGG_H */

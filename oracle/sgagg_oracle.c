/*
 * sgagg_oracle.c -- plain, slow, obviously correct CPU oracle for sort-based
 * grouping and aggregation (Do, Graefe, Naughton, "Efficient sorting,
 * duplicate removal, grouping, and aggregation", arXiv 2010.00152).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code with the CUDA path.
 *
 * What it computes (Sec. 1, the "select ..., count(*), sum(X), min(Z) ...
 * group by A, B" statement of the problem; Sec. 3.3 on intermediate rows that
 * carry sums and counts; Sec. 6.1 on in-stream aggregation and sorted output):
 * one output row per distinct normalized key, keys strictly ascending as
 * unsigned integers, and per requested aggregate
 *   COUNT = number of input rows with that key,
 *   SUM   = sum of the payload column modulo 2^64 (reported as int64),
 *   MIN   = signed minimum, MAX = signed maximum.
 * The method is exact, so the plain definition is the oracle: sort the
 * (key, row) pairs, then fold runs of equal keys in one in-stream pass.
 * Integer +, min and max are associative and commutative (sums are taken in
 * uint64 so that overflow wraps), so the result is unique.
 *
 * Also here: the run-generation step alone (read-sort-write cycles with early
 * aggregation, Sec. 3 and Sec. 6.1) and the merge of runs of partial
 * aggregates (Sec. 4), each written the plain way, so that tests can check the
 * run bookkeeping of the GPU path (rows per run) exactly.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_COUNT = 0, ORC_SUM = 1, ORC_MIN = 2, ORC_MAX = 3 };

/* ------------------------------------------------------------------------ */
/* Normalized keys (Sec. 2.4, "normalized keys encode key values in          */
/* order-preserving strings"): unsigned key columns concatenated, column 0   */
/* most significant, so that comparing the integers compares the tuples      */
/* lexicographically.  Returns 0, or -1 if the widths add up to more than 64 */
/* bits or a width is not 1, 2, 4 or 8 bytes.                               */
/* ------------------------------------------------------------------------ */
int orc_normalize(int n_cols, const int32_t *bytes, const void *const *cols,
                  int64_t n, uint64_t *out)
{
    int total = 0;
    for (int c = 0; c < n_cols; ++c) {
        int b = bytes[c];
        if (b != 1 && b != 2 && b != 4 && b != 8) return -1;
        total += 8 * b;
    }
    if (n_cols < 1 || total > 64) return -1;
    for (int64_t i = 0; i < n; ++i) {
        uint64_t k = 0;
        for (int c = 0; c < n_cols; ++c) {
            uint64_t v;
            switch (bytes[c]) {
            case 1: v = ((const uint8_t *)cols[c])[i]; break;
            case 2: v = ((const uint16_t *)cols[c])[i]; break;
            case 4: v = ((const uint32_t *)cols[c])[i]; break;
            default: v = ((const uint64_t *)cols[c])[i]; break;
            }
            /* shift the previous columns up by this column's width */
            k = (bytes[c] == 8) ? v : ((k << (8 * bytes[c])) | v);
        }
        out[i] = k;
    }
    return 0;
}

/* Inverse of orc_normalize for one column: the bits of column c. */
void orc_unpack(int n_cols, const int32_t *bytes, int c, const uint64_t *keys,
                int64_t n, void *out)
{
    int below = 0; /* bits of the columns after c */
    for (int j = c + 1; j < n_cols; ++j) below += 8 * bytes[j];
    for (int64_t i = 0; i < n; ++i) {
        uint64_t v = (below >= 64) ? 0 : (keys[i] >> below);
        switch (bytes[c]) {
        case 1: ((uint8_t *)out)[i] = (uint8_t)v; break;
        case 2: ((uint16_t *)out)[i] = (uint16_t)v; break;
        case 4: ((uint32_t *)out)[i] = (uint32_t)v; break;
        default: ((uint64_t *)out)[i] = v; break;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Group by on raw rows: sort, then in-stream aggregation.                   */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; int64_t row; } orc_pair;

static int orc_cmp_pair(const void *pa, const void *pb)
{
    const orc_pair *a = (const orc_pair *)pa, *b = (const orc_pair *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->row > b->row) - (a->row < b->row);
}

/* Value an input row contributes to aggregate `op` over payload column v. */
static int64_t orc_init_value(int op, int64_t v) { return op == ORC_COUNT ? 1 : v; }

/* Row-plus-row accumulation (Sec. 6.1): combine two partial aggregates. */
static int64_t orc_combine(int op, int64_t acc, int64_t v)
{
    switch (op) {
    case ORC_COUNT:
    case ORC_SUM: return (int64_t)((uint64_t)acc + (uint64_t)v);
    case ORC_MIN: return v < acc ? v : acc;
    default:      return v > acc ? v : acc;
    }
}

/*
 * keys[n] normalized keys; pay[c][n] int64 payload columns; aggregate a is
 * (ops[a], cols[a]) with cols[a] ignored for COUNT.  out_keys / out_aggs[a]
 * must have room for n rows.  Returns the number of groups, or -1 on a bad
 * argument or allocation failure.
 */
int64_t orc_groupby(const uint64_t *keys, int64_t n, int n_pay,
                    const int64_t *const *pay, int n_aggs, const int32_t *ops,
                    const int32_t *cols, uint64_t *out_keys, int64_t *const *out_aggs)
{
    for (int a = 0; a < n_aggs; ++a) {
        if (ops[a] < ORC_COUNT || ops[a] > ORC_MAX) return -1;
        if (ops[a] != ORC_COUNT && (cols[a] < 0 || cols[a] >= n_pay)) return -1;
    }
    if (n <= 0) return 0;
    orc_pair *p = (orc_pair *)malloc((size_t)n * sizeof(orc_pair));
    if (!p) return -1;
    for (int64_t i = 0; i < n; ++i) { p[i].key = keys[i]; p[i].row = i; }
    qsort(p, (size_t)n, sizeof(orc_pair), orc_cmp_pair);

    int64_t g = -1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t r = p[i].row;
        int fresh = (i == 0) || (p[i].key != p[i - 1].key);
        if (fresh) { ++g; out_keys[g] = p[i].key; }
        for (int a = 0; a < n_aggs; ++a) {
            int64_t v = orc_init_value(ops[a], ops[a] == ORC_COUNT ? 0 : pay[cols[a]][r]);
            out_aggs[a][g] = fresh ? v : orc_combine(ops[a], out_aggs[a][g], v);
        }
    }
    free(p);
    return g + 1;
}

/*
 * Fold rows that already carry partial aggregates (the row format of runs,
 * Sec. 3.3): state[a][n] holds aggregate a of each row.  Same output contract
 * as orc_groupby.  Used for the merge of runs (Sec. 4): the final output is the
 * fold of the union of all runs.
 */
int64_t orc_fold_states(const uint64_t *keys, int64_t n, int n_aggs,
                        const int32_t *ops, const int64_t *const *state,
                        uint64_t *out_keys, int64_t *const *out_aggs)
{
    if (n <= 0) return 0;
    orc_pair *p = (orc_pair *)malloc((size_t)n * sizeof(orc_pair));
    if (!p) return -1;
    for (int64_t i = 0; i < n; ++i) { p[i].key = keys[i]; p[i].row = i; }
    qsort(p, (size_t)n, sizeof(orc_pair), orc_cmp_pair);
    int64_t g = -1;
    for (int64_t i = 0; i < n; ++i) {
        int64_t r = p[i].row;
        int fresh = (i == 0) || (p[i].key != p[i - 1].key);
        if (fresh) { ++g; out_keys[g] = p[i].key; }
        for (int a = 0; a < n_aggs; ++a) {
            int64_t v = state[a][r];
            out_aggs[a][g] = fresh ? v : orc_combine(ops[a], out_aggs[a][g], v);
        }
    }
    free(p);
    return g + 1;
}

/*
 * Run generation with early aggregation by read-sort-write cycles (Sec. 3;
 * Sec. 6.1: "the size of initial runs equals the memory size"): the input is
 * cut into batches of M consecutive rows (the last one shorter); each batch is
 * sorted and its equal keys folded before the run is written.  Run b is
 * appended to run_keys / run_state[a] (capacity n rows each) and its row count
 * stored in run_rows[b] (capacity ceil(n/M)).  Returns the number of runs, or
 * -1 on a bad argument.
 */
int64_t orc_run_generation(const uint64_t *keys, int64_t n, int64_t M, int n_pay,
                           const int64_t *const *pay, int n_aggs, const int32_t *ops,
                           const int32_t *cols, int64_t *run_rows, uint64_t *run_keys,
                           int64_t *const *run_state)
{
    if (M < 1 || n < 0 || n_aggs > 64) return -1;
    int64_t runs = 0, at = 0;
    const int64_t *bpay[64];
    int64_t *bstate[64];
    for (int64_t s = 0; s < n; s += M) {
        int64_t m = (n - s < M) ? (n - s) : M;
        for (int c = 0; c < n_pay && c < 64; ++c) bpay[c] = pay[c] + s;
        for (int a = 0; a < n_aggs; ++a) bstate[a] = run_state[a] + at;
        int64_t g = orc_groupby(keys + s, m, n_pay, bpay, n_aggs, ops, cols,
                                run_keys + at, bstate);
        if (g < 0) return -1;
        run_rows[runs++] = g;
        at += g;
    }
    return runs;
}

/*
 * Run generation with an absorbing in-memory index (Sec. 3 on early
 * aggregation: key values equal to ones already in the index are absorbed by
 * aggregation; Sec. 6.1 on the in-sort aggregation algorithm: each input
 * batch is sorted first to detect duplicates within the batch, only the
 * batch's distinct keys are looked up in the ordered index, and when memory
 * runs out the index is written as a sorted run, read-sort-write style, so
 * that runs hold M keys).
 *
 * The index is a sorted array of at most M distinct keys with their partial
 * aggregates.  Batch by batch (B consecutive input rows, the last shorter):
 * the batch is grouped (sorted, equal keys folded); its distinct keys are
 * then taken in ascending order -- a key already in the index is absorbed
 * (aggregates combined); a new key is inserted while the index holds fewer
 * than M keys; otherwise the whole index is written as a run, emptied, and
 * the key inserted.  At the end, if no run was written the index is the
 * output; else it is written as the last run.
 *
 * run_rows[] (capacity n + 1) receives every run's row count; returns the
 * number of runs (0: the input was absorbed in memory), or -1 on a bad
 * argument or allocation failure.  *index_rows receives the rows left in the
 * index at the end (the output rows when no run was written).
 */
int64_t orc_absorb_runs(const uint64_t *keys, int64_t n, int64_t M, int64_t B, int n_pay,
                        const int64_t *const *pay, int n_aggs, const int32_t *ops,
                        const int32_t *cols, int64_t *run_rows, int64_t *index_rows)
{
    if (M < 1 || B < 1 || n < 0 || n_aggs > 64) return -1;
    const size_t A = (size_t)(n_aggs > 0 ? n_aggs : 1);
    /* the index (old) and the index being rebuilt while the batch's keys are
       taken in ascending order (new); inserting keys in ascending order into
       a sorted array is a merge of the two sorted lists */
    uint64_t *ok = (uint64_t *)malloc((size_t)M * sizeof(uint64_t));
    uint64_t *nk = (uint64_t *)malloc((size_t)M * sizeof(uint64_t));
    int64_t *os = (int64_t *)malloc((size_t)M * A * sizeof(int64_t));
    int64_t *ns = (int64_t *)malloc((size_t)M * A * sizeof(int64_t));
    int64_t bmax = B < n ? B : (n > 0 ? n : 1);
    uint64_t *bk = (uint64_t *)malloc((size_t)bmax * sizeof(uint64_t));
    int64_t *bsd = (int64_t *)malloc((size_t)bmax * A * sizeof(int64_t));
    if (!ok || !nk || !os || !ns || !bk || !bsd) {
        free(ok); free(nk); free(os); free(ns); free(bk); free(bsd);
        return -1;
    }
    int64_t r = 0, runs = 0;
    const int64_t *bpay[64];
    int64_t *bst[64];
    for (int a = 0; a < n_aggs; ++a) bst[a] = bsd + (size_t)a * (size_t)bmax;
    for (int64_t s = 0; s < n; s += B) {
        int64_t m = (n - s < B) ? (n - s) : B;
        for (int c = 0; c < n_pay && c < 64; ++c) bpay[c] = pay[c] + s;
        int64_t g = orc_groupby(keys + s, m, n_pay, bpay, n_aggs, ops, cols, bk, bst);
        if (g < 0) { free(ok); free(nk); free(os); free(ns); free(bk); free(bsd); return -1; }
        int64_t i = 0, w = 0;  /* next old entry, entries in the new index */
        for (int64_t j = 0; j < g; ++j) {
            const uint64_t x = bk[j];
            while (i < r && ok[i] < x) {  /* old keys below x stay */
                nk[w] = ok[i];
                for (int a = 0; a < n_aggs; ++a) ns[(size_t)a * (size_t)M + (size_t)w] = os[(size_t)a * (size_t)M + (size_t)i];
                ++w; ++i;
            }
            if (i < r && ok[i] == x) {  /* absorbed */
                for (int a = 0; a < n_aggs; ++a)
                    os[(size_t)a * (size_t)M + (size_t)i] =
                        orc_combine(ops[a], os[(size_t)a * (size_t)M + (size_t)i], bst[a][j]);
                continue;
            }
            if (w + (r - i) == M) {  /* memory full: the index becomes a run */
                run_rows[runs++] = M;
                w = 0;
                i = r = 0;
            }
            nk[w] = x;  /* inserted */
            for (int a = 0; a < n_aggs; ++a) ns[(size_t)a * (size_t)M + (size_t)w] = bst[a][j];
            ++w;
        }
        while (i < r) {  /* old keys above the batch's last key */
            nk[w] = ok[i];
            for (int a = 0; a < n_aggs; ++a) ns[(size_t)a * (size_t)M + (size_t)w] = os[(size_t)a * (size_t)M + (size_t)i];
            ++w; ++i;
        }
        uint64_t *tk = ok; ok = nk; nk = tk;
        int64_t *ts = os; os = ns; ns = ts;
        r = w;
    }
    if (runs > 0) run_rows[runs++] = r;
    *index_rows = r;
    free(ok); free(nk); free(os); free(ns); free(bk); free(bsd);
    return runs;
}

/*
 * count(distinct u) per group g, with the other aggregates over all rows of
 * g (the duplicate removal followed by grouping of Sec. 7, Hypothesis 6):
 * the plain definition -- sort the (g, u, row) triples, walk them once; a
 * new g opens an output row, a new (g, u) pair adds one distinct value, and
 * every row is folded into its g.  gkeys are normalized group keys, ukeys
 * the distinct column.  out_distinct[g] receives the distinct count.
 * Returns the number of groups, or -1 on a bad argument.
 */
typedef struct { uint64_t g, u; int64_t row; } orc_triple;

static int orc_cmp_triple(const void *pa, const void *pb)
{
    const orc_triple *a = (const orc_triple *)pa, *b = (const orc_triple *)pb;
    if (a->g != b->g) return a->g < b->g ? -1 : 1;
    if (a->u != b->u) return a->u < b->u ? -1 : 1;
    return (a->row > b->row) - (a->row < b->row);
}

int64_t orc_count_distinct(const uint64_t *gkeys, const uint64_t *ukeys, int64_t n, int n_pay,
                           const int64_t *const *pay, int n_aggs, const int32_t *ops, const int32_t *cols,
                           uint64_t *out_keys, int64_t *out_distinct, int64_t *const *out_aggs)
{
    for (int a = 0; a < n_aggs; ++a) {
        if (ops[a] < ORC_COUNT || ops[a] > ORC_MAX) return -1;
        if (ops[a] != ORC_COUNT && (cols[a] < 0 || cols[a] >= n_pay)) return -1;
    }
    if (n <= 0) return 0;
    orc_triple *t = (orc_triple *)malloc((size_t)n * sizeof(orc_triple));
    if (!t) return -1;
    for (int64_t i = 0; i < n; ++i) { t[i].g = gkeys[i]; t[i].u = ukeys[i]; t[i].row = i; }
    qsort(t, (size_t)n, sizeof(orc_triple), orc_cmp_triple);
    int64_t g = -1;
    for (int64_t i = 0; i < n; ++i) {
        const int new_g = (i == 0) || (t[i].g != t[i - 1].g);
        const int new_u = new_g || (t[i].u != t[i - 1].u);
        if (new_g) { ++g; out_keys[g] = t[i].g; out_distinct[g] = 0; }
        if (new_u) ++out_distinct[g];
        for (int a = 0; a < n_aggs; ++a) {
            int64_t v = orc_init_value(ops[a], ops[a] == ORC_COUNT ? 0 : pay[cols[a]][t[i].row]);
            out_aggs[a][g] = new_g ? v : orc_combine(ops[a], out_aggs[a][g], v);
        }
    }
    free(t);
    return g + 1;
}

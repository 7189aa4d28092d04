"""The paper's analytic spill model (arXiv 2010.00152, Sec. 3.4, 4, 5.2).

TEST INFRASTRUCTURE ONLY.  Sizes are in rows, as in the paper's examples.
Every function states the passage it restates; tests pin each one to the
numbers the paper prints (Examples 2-5, the hybrid example of Sec. 5.2.3).

Also here: the expected number of distinct keys in a batch of rows drawn
uniformly from D values (the classic occupancy problem), which predicts the
size of a run produced by read-sort-write run generation with early
aggregation when keys are uniform.
"""
import math


def runs_read_sort_write(I, M):
    """Read-sort-write cycles make runs the size of memory (Sec. 3, Sec. 6.1)."""
    return -(-I // M)


def runs_replacement_selection(I, M):
    """Replacement selection: expected run count I/(2M) + 1 (Sec. 5.2.2)."""
    return I / (2 * M) + 1


def absorb_probability(M, O):
    """Chance an input row finds its key in a full in-memory index (Sec. 3.4)."""
    return min(1.0, M / O)


def early_agg_initial_run_volume(I, M, O):
    """Total size of initial runs with early aggregation and memory always
    full: M + (1 - M/O) * I for O > M (Example 2, Sec. 3.2); no spill at all
    when the output fits in memory (Table of conditions for in-memory
    operation, Sec. 5.2.1)."""
    if O <= M:
        return 0.0
    return M + (1.0 - M / O) * I


def in_memory(method, I, O, M):
    """Condition for an in-memory operation (Sec. 5.2.1 table)."""
    if method in ("hash", "new_in_sort"):
        return O <= M
    if method in ("sort_separate", "sort_traditional_early"):
        return I <= M
    raise ValueError(method)


def levels(x, F):
    """Smallest integer L >= 0 with F**L >= x (merge / partitioning levels)."""
    L, p = 0, 1
    while p < x:
        p *= F
        L += 1
    return L


def spill_volume(method, I, O, M, F, replacement_selection=False):
    """Total spill volume of the Sec. 5.2.2 table (rows written to temporary
    storage, each later read once), with the logarithms rounded up to whole
    levels."""
    if method == "hash":
        return levels(O / M, F) * I
    if method == "sort_separate":
        x = (1 + I / (2 * M)) if replacement_selection else I / M
        return levels(x, F) * I
    if method == "sort_traditional_early":
        return levels(O / M, F) * I + (I - O) / (F - 1)
    if method == "new_in_sort":
        x = (1 + O / (2 * M)) if replacement_selection else O / M
        return levels(x, F) * I
    raise ValueError(method)


def merge_levels_then_steps(run_sizes, F, O):
    """Traditional merging with aggregation inside runs, as worked through in
    Example 3 (Sec. 4.1): full merge levels (consecutive groups of F runs),
    each merged run capped at the final output size O by early duplicate
    removal; once runs reach O, single merge steps of fan-in
    min(F, k - F + 1) until at most F runs remain for the final merge.

    Returns (rows written by intermediate merges, run counts after each
    level or step)."""
    runs = list(run_sizes)
    spilled, counts = 0.0, []
    while len(runs) > F:
        if max(runs) < O:
            runs = [min(sum(runs[i:i + F]), O) for i in range(0, len(runs), F)]
            spilled += sum(runs)
        else:
            runs.sort()
            f = min(F, len(runs) - F + 1)
            merged = min(sum(runs[:f]), O)
            runs = runs[f:] + [merged]
            spilled += merged
        counts.append(len(runs))
    return spilled, counts


def merge_steps_smallest_first(run_sizes, F, O):
    """Traditional merge steps as in the footnote to Example 4 (Sec. 4.2): a
    first step of fan-in ((k - 1) mod (F - 1)) + 1, then steps of fan-in F,
    always merging the smallest runs, each output capped at O, until F runs
    remain for the final merge step.

    Returns (rows written by intermediate merges, run counts after each step)."""
    runs = sorted(run_sizes)
    spilled, counts = 0.0, []
    first = True
    while len(runs) > F:
        f = ((len(runs) - 1) % (F - 1)) + 1 if first else F
        if f == 1:
            f = F
        first = False
        merged = min(sum(runs[:f]), O)
        runs = sorted(runs[f:] + [merged])
        spilled += merged
        counts.append(len(runs))
    return spilled, counts


def hybrid_fanout(O, M, P):
    """Actual fan-out/fan-in of a hybrid algorithm, f = ceil((O - M)/(M - P))
    (Sec. 5.2.3 table), clamped below at 0 (in-memory case)."""
    return max(0, math.ceil((O - M) / (M - P)))


def merge_steps_full_levels(k, F):
    """Merge steps and levels needed to reduce k runs to one with fan-in F,
    merging whole levels (Sec. 5.2.3: 1,000 runs and F = 10 take three levels
    and 111 steps)."""
    steps = lvls = 0
    while k > 1:
        nxt = -(-k // F)
        steps += nxt
        lvls += 1
        k = nxt
    return steps, lvls


def expected_distinct(b, D):
    """Expected number of distinct values among b draws uniform over D values:
    D * (1 - (1 - 1/D)**b) (occupancy problem)."""
    return D * (1.0 - (1.0 - 1.0 / D) ** b)


def var_distinct(b, D):
    """Variance of the number of distinct values among b uniform draws over D
    values: D q1 + D (D - 1) q2 - D^2 q1^2 with q1 = (1 - 1/D)^b,
    q2 = (1 - 2/D)^b (occupancy problem)."""
    q1 = (1.0 - 1.0 / D) ** b
    q2 = (1.0 - 2.0 / D) ** b
    return D * q1 + D * (D - 1) * q2 - D * D * q1 * q1


def expected_run_rows(n, M, D):
    """Expected total rows of all runs written by read-sort-write run
    generation with early aggregation over n rows with keys uniform over D
    values and batches of M rows: the sum over batches of the expected
    distinct keys per batch."""
    tot, var, s = 0.0, 0.0, 0
    while s < n:
        b = min(M, n - s)
        tot += expected_distinct(b, D)
        var += var_distinct(b, D)
        s += b
    return tot, var

"""Trend counts, the approximate-trend threshold and the fitness of one individual.

Definition followed (Sec. 2.3, "EBIC" paragraph; Sec. 2.4, steps 2-3 and the parameter list):
an individual is a series of columns c_0..c_{L-1}; the series defines an increasing order that
the values of every row of the bicluster must follow.  For a row r:

    inc_r = #{k < L-1 : x[r, c_{k+1}] > x[r, c_k]}      (positive trend pairs)
    dec_r = #{k < L-1 : x[r, c_{k+1}] < x[r, c_k]}      (negative trend pairs)

Readings where the paper is silent:
  * ties break both trends (strict comparisons of the float32 values; -0 equals +0);
  * consecutive pairs of the series are counted;
  * approximate threshold t(L) = ceil(ratio * (L-1)) in exact integer arithmetic, so ratio 1/1 is
    the exact trend and L = 2 needs its single pair;
  * with negative trends on, a row is accepted when it passes either direction (counted once);
  * fitness f = 0 when fewer than ``min_rows`` rows are accepted or the individual is dead, else
    rows_any * 2**min(L, col_cap), an exact integer.

Two variants of the pair test, each a flag (both off by default):
  * ``non_strict``: a positive pair holds when x[r, c_{k+1}] >= x[r, c_k] and a negative pair when
    x[r, c_{k+1}] <= x[r, c_k], so a tie counts for both directions;
  * ``last_kept``: each direction compares a value with the last value that kept the trend rather
    than with its predecessor: last = x[r, c_0]; for k = 1..L-1, when the pair (last, x[r, c_k])
    holds the count grows and last becomes x[r, c_k]; a value that breaks the trend is skipped.
    With the exact threshold (every pair) both ways of counting accept the same rows.

Test infrastructure only (see the package docstring).
"""

import numpy as np


def threshold(L, ratio_num, ratio_den):
    """t(L) = ceil(ratio_num * (L-1) / ratio_den)."""
    pairs = L - 1
    return (ratio_num * pairs + ratio_den - 1) // ratio_den


def check_matrix(x):
    x = np.asarray(x)
    if x.ndim != 2 or x.dtype != np.float32:
        raise ValueError("matrix must be a 2-D float32 array")
    if not np.isfinite(x).all():
        raise ValueError("matrix holds NaN or Inf")
    return x


def check_chromosome(cols, n_cols):
    cols = [int(c) for c in cols]
    if not (2 <= len(cols) <= 64):
        raise ValueError("chromosome length must be in [2, 64]")
    if len(set(cols)) != len(cols) or min(cols) < 0 or max(cols) >= n_cols:
        raise ValueError("chromosome columns must be distinct and in range")
    return cols


def pair_holds(nxt, prev, positive, non_strict):
    """The pair test of one direction (element-wise over rows)."""
    if positive:
        return nxt >= prev if non_strict else nxt > prev
    return nxt <= prev if non_strict else nxt < prev


def trend_count(sub, positive, non_strict, last_kept):
    """Per-row count of the series' pairs that follow the direction (sub = R x L values)."""
    if not last_kept:
        return pair_holds(sub[:, 1:], sub[:, :-1], positive, non_strict).sum(axis=1)
    last = sub[:, 0].copy()
    count = np.zeros(sub.shape[0], dtype=np.int64)
    for k in range(1, sub.shape[1]):
        hit = pair_holds(sub[:, k], last, positive, non_strict)
        count += hit
        last = np.where(hit, sub[:, k], last)
    return count


def row_trend_masks(x, cols, neg_trends, ratio_num, ratio_den, non_strict=0, last_kept=0):
    """Boolean masks over rows: (pos_ok, neg_ok) for one individual, from the plain definition."""
    sub = x[:, cols]                       # R x L, float32
    inc = trend_count(sub, True, non_strict, last_kept)
    dec = trend_count(sub, False, non_strict, last_kept)
    t = threshold(len(cols), ratio_num, ratio_den)
    pos_ok = inc >= t
    neg_ok = (dec >= t) if neg_trends else np.zeros_like(pos_ok)
    return pos_ok, neg_ok


def fitness(rows_any, L, min_rows, col_cap, dead=False):
    if dead or rows_any < min_rows:
        return 0
    return int(rows_any) << min(int(L), int(col_cap))


def eval_individual(x, cols, p):
    pos_ok, neg_ok = row_trend_masks(x, cols, p.neg_trends, p.ratio_num, p.ratio_den,
                                     p.non_strict, p.last_kept)
    rp = int(pos_ok.sum())
    rn = int(neg_ok.sum())
    ra = int((pos_ok | neg_ok).sum())
    return rp, rn, ra, fitness(ra, len(cols), p.min_rows, p.col_cap)


def eval_population(x, col_idx, offsets, p):
    """Counts and fitness for a CSR population (col_idx[offsets[i]:offsets[i+1]] = individual i).

    Returns four int64 arrays rows_pos, rows_neg, rows_any, fitness."""
    x = check_matrix(x)
    n = len(offsets) - 1
    out = np.zeros((4, n), dtype=np.int64)
    for i in range(n):
        cols = check_chromosome(col_idx[offsets[i]:offsets[i + 1]], x.shape[1])
        out[:, i] = eval_individual(x, cols, p)
    return out[0], out[1], out[2], out[3].astype(np.uint64)

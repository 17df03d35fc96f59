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


def row_trend_masks(x, cols, neg_trends, ratio_num, ratio_den):
    """Boolean masks over rows: (pos_ok, neg_ok) for one individual, from the plain definition."""
    sub = x[:, cols]                       # R x L, float32
    nxt, cur = sub[:, 1:], sub[:, :-1]
    inc = (nxt > cur).sum(axis=1)
    dec = (nxt < cur).sum(axis=1)
    t = threshold(len(cols), ratio_num, ratio_den)
    pos_ok = inc >= t
    neg_ok = (dec >= t) if neg_trends else np.zeros_like(pos_ok)
    return pos_ok, neg_ok


def fitness(rows_any, L, min_rows, col_cap, dead=False):
    if dead or rows_any < min_rows:
        return 0
    return int(rows_any) << min(int(L), int(col_cap))


def eval_individual(x, cols, p):
    pos_ok, neg_ok = row_trend_masks(x, cols, p.neg_trends, p.ratio_num, p.ratio_den)
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

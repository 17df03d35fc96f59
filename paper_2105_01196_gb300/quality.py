"""Clustering error (CE, Eq. 1 of the EBIC.jl paper) of found biclusters against a reference set.

A host-side measure of a finished run's result (it is not a step of the device path): each
bicluster is the rectangle of matrix cells rows x columns.  The confusion entry of found
bicluster i and reference bicluster j is |rows_i & rows_j| * |cols_i & cols_j| (the cells two
rectangles share), D_max is the largest total over one-to-one assignments (Munkres / Hungarian
algorithm, here scipy's linear_sum_assignment), and U is the union of all cells of both sets.
The paper prints CE = (|U| - D_max) / |U| but describes it as a goodness of fit with 1 for a
perfect match; ``error`` is the printed value and ``score`` = D_max / |U| = 1 - error the
described one.
"""

import numpy as np


def _as_sets(biclusters):
    out = []
    for rows, cols in biclusters:
        out.append((np.unique(np.asarray(rows, dtype=np.int64)),
                    np.unique(np.asarray(cols, dtype=np.int64))))
    return out


def rows_from_mask(words, n_rows):
    """Row indices set in a row mask of uint32 words (bit j of word w = row 32 w + j)."""
    w = np.asarray(words, dtype=np.uint32)
    bits = ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(bool).reshape(-1)
    return np.nonzero(bits[:n_rows])[0]


def clustering_error(found, reference, n_rows, n_cols):
    """Returns dict(d_max, union, error, score) for lists of (rows, cols) biclusters."""
    from scipy.optimize import linear_sum_assignment

    f = _as_sets(found)
    r = _as_sets(reference)
    covered = np.zeros((n_rows, n_cols), dtype=bool)
    for rows, cols in f + r:
        covered[np.ix_(rows, cols)] = True
    union = int(covered.sum())
    d = 0
    if f and r:
        m = np.zeros((len(f), len(r)), dtype=np.int64)
        for i, (ri, ci) in enumerate(f):
            for j, (rj, cj) in enumerate(r):
                m[i, j] = (len(np.intersect1d(ri, rj, assume_unique=True)) *
                           len(np.intersect1d(ci, cj, assume_unique=True)))
        a, b = linear_sum_assignment(m, maximize=True)
        d = int(m[a, b].sum())
    if union == 0:
        return {"d_max": 0, "union": 0, "error": 0.0, "score": 1.0}
    return {"d_max": d, "union": union, "error": (union - d) / union, "score": d / union}

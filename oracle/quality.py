"""Clustering error (CE) between two sets of biclusters (Eq. 1, "Performance measure" paragraph
of the EBIC.jl paper's experimental section).

TEST INFRASTRUCTURE ONLY (see the package docstring).

A bicluster is the set of matrix cells (r, c) with r in its rows and c in its columns.  The
confusion entry of a detected bicluster i and a true bicluster j is the number of cells they
share.  D_max is the largest sum of confusion entries over one-to-one assignments between the two
sets (the paper finds it with the Munkres algorithm), and U is the union of the cells of all
biclusters of both sets.  Eq. 1 prints (|U| - D_max) / |U|, while the text calls CE a goodness of
fit where 1 is a perfect match; the reading taken here reports both: ``error`` follows the printed
formula (0 = identical) and ``score`` = D_max / |U| = 1 - error follows the text.

This version is written for checking by eye: cells as Python sets, and D_max by trying every
one-to-one assignment (only for small sets).
"""

from fractions import Fraction
from itertools import permutations


def cells(rows, cols):
    """The cell set of a bicluster."""
    return {(int(r), int(c)) for r in rows for c in cols}


def confusion(detected, truth):
    """M[i][j] = |cells(detected[i]) & cells(truth[j])|; each bicluster is (rows, cols)."""
    det = [cells(r, c) for r, c in detected]
    tru = [cells(r, c) for r, c in truth]
    return [[len(a & b) for b in tru] for a in det]


def d_max(m):
    """Largest sum over one-to-one assignments of rows to columns of m (brute force)."""
    n_det = len(m)
    n_tru = len(m[0]) if n_det else 0
    if n_det == 0 or n_tru == 0:
        return 0
    best = 0
    if n_det <= n_tru:
        for perm in permutations(range(n_tru), n_det):
            best = max(best, sum(m[i][perm[i]] for i in range(n_det)))
    else:
        for perm in permutations(range(n_det), n_tru):
            best = max(best, sum(m[perm[j]][j] for j in range(n_tru)))
    return best


def union_size(detected, truth):
    u = set()
    for r, c in list(detected) + list(truth):
        u |= cells(r, c)
    return len(u)


def clustering_error(detected, truth):
    """(D_max, |U|, error, score) with error = (|U| - D_max) / |U| and score = D_max / |U| as
    exact fractions (both 0 / 1 conventions: an empty union gives error 0, score 1)."""
    m = confusion(detected, truth)
    d = d_max(m)
    u = union_size(detected, truth)
    if u == 0:
        return 0, 0, Fraction(0), Fraction(1)
    return d, u, Fraction(u - d, u), Fraction(d, u)

"""Clustering error (CE, Eq. 1): the oracle's brute-force form pinned by hand-worked examples, the
package's Munkres form against it, and the search's CE on an easy planted matrix."""

from fractions import Fraction

import numpy as np
import pytest

from oracle import ebic
from oracle.params import Params
from oracle.quality import clustering_error as ce_oracle
from paper_2105_01196_gb300 import synth
from paper_2105_01196_gb300.quality import clustering_error as ce_package, rows_from_mask


def rect(r0, r1, cols):
    return (list(range(r0, r1)), list(cols))


def test_hand_example_where_greedy_assignment_is_wrong():
    # Truth A = rows 0-4 x col 0 (5 cells), B = rows 0-3 x col 1 (4 cells).
    # Found X = rows 0-4 x cols 0,1 (10 cells: 5 shared with A, 4 with B),
    #       Y = rows 0-3 x col 0 (4 cells: 4 shared with A, 0 with B).
    # Greedy X-A, Y-B gives 5; the optimal assignment X-B, Y-A gives 8.  Every cell lies in X,
    # so |U| = 10: error 2/10, score 8/10.
    truth = [rect(0, 5, [0]), rect(0, 4, [1])]
    found = [rect(0, 5, [0, 1]), rect(0, 4, [0])]
    d, u, err, score = ce_oracle(found, truth)
    assert (d, u) == (8, 10)
    assert err == Fraction(1, 5) and score == Fraction(4, 5)


def test_identical_disjoint_and_partial():
    a = [rect(0, 10, [0, 1, 2]), rect(20, 25, [5, 6])]
    assert ce_oracle(a, a)[2:] == (Fraction(0), Fraction(1))
    b = [rect(30, 40, [7, 8])]
    d, u, err, score = ce_oracle(a, b)
    assert d == 0 and u == 30 + 10 + 20 and score == 0
    # half of the rows of a single bicluster: 5 x 3 shared cells, union 10 x 3
    d, u, _, score = ce_oracle([rect(0, 5, [0, 1, 2])], [rect(0, 10, [0, 1, 2])])
    assert (d, u, score) == (15, 30, Fraction(1, 2))


def test_unequal_numbers_of_biclusters():
    # three found against one true: only the best one is assigned, all count in the union
    truth = [rect(0, 4, [0, 1])]                                   # 8 cells
    found = [rect(0, 2, [0, 1]), rect(0, 4, [0, 1]), rect(6, 7, [3])]
    d, u, _, score = ce_oracle(found, truth)
    assert (d, u) == (8, 9) and score == Fraction(8, 9)


def test_order_and_role_invariance():
    g = np.random.default_rng(1)
    for _ in range(20):
        sets = []
        for _ in range(int(g.integers(1, 5))):
            r0 = int(g.integers(0, 20))
            sets.append((list(range(r0, r0 + int(g.integers(1, 8)))),
                         sorted(g.choice(10, size=int(g.integers(1, 4)), replace=False).tolist())))
        k = int(g.integers(0, len(sets) + 1))
        found, truth = sets[:k], sets[k:]
        base = ce_oracle(found, truth)
        assert ce_oracle(found[::-1], truth[::-1]) == base
        assert ce_oracle(truth, found) == base
        assert 0 <= base[3] <= 1


def test_package_munkres_matches_oracle():
    g = np.random.default_rng(7)
    for _ in range(60):
        def one():
            rows = np.sort(g.choice(40, size=int(g.integers(1, 15)), replace=False))
            cols = np.sort(g.choice(12, size=int(g.integers(1, 6)), replace=False))
            return rows.tolist(), cols.tolist()
        found = [one() for _ in range(int(g.integers(0, 6)))]
        truth = [one() for _ in range(int(g.integers(0, 6)))]
        d, u, err, score = ce_oracle(found, truth)
        got = ce_package(found, truth, 40, 12)
        assert (got["d_max"], got["union"]) == (d, u)
        assert got["score"] == pytest.approx(float(score), abs=0.0)


def test_rows_from_mask():
    words = np.array([0b1011, 1 << 31, 1], dtype=np.uint32)
    assert rows_from_mask(words, 70).tolist() == [0, 1, 3, 63, 64]
    assert rows_from_mask(words, 64).tolist() == [0, 1, 3, 63]


def test_search_ce_on_an_easy_planted_matrix():
    """The oracle search (Sec. 2.4) on 40 planted rows x 4 columns of a 160 x 10 N(0,1) matrix:
    the best top-list entry, with the rows that follow it, matches the planted bicluster with
    CE score >= 0.8 (the background rows that follow 4 columns by chance, about 160/24, are the
    only loss)."""
    x, truth = synth.planted_matrix(160, 10, 1, (40, 40), (4, 4), seed=77, neg_fraction=0.0)
    p = Params(neg_trends=0, ratio_num=1, ratio_den=1, max_len=5, init_min_len=2, init_max_len=4,
               pop_size=48, elite=4, n_biclusters=4, tabu_hit_limit=0, seed=4)
    st = ebic.run(x, p, 40)
    masks = ebic.extract(x, st, p)
    ridx, order, _ = truth[0]
    found = [(rows_from_mask(masks[0], x.shape[0]), list(st.top[0].cols))]
    assert set(found[0][1]) == set(int(c) for c in order)
    d, u, _, score = ce_oracle(found, [(ridx, order)])
    assert score >= Fraction(4, 5)
    got = ce_package(found, [(ridx, order)], *x.shape)
    assert (got["d_max"], got["union"]) == (d, u)

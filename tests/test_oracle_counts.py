"""Pins of the oracle's trend counts, threshold, fitness and pair bitmap (no GPU).

Each test checks the oracle against something other than itself: a hand-worked example of the
trend definition (Sec. 2.3), brute force over every column sequence of a tiny matrix, invariants
the definition implies, closed forms of the threshold, and an independent per-row loop."""

import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import counts
from oracle.bitmap import pair_bitmap, pair_words
from oracle.params import Params
from paper_2105_01196_gb300 import synth


def P(**kw):
    base = dict(neg_trends=1, ratio_num=1, ratio_den=1, min_rows=0, col_cap=10)
    base.update(kw)
    return Params(**base)


def masks(x, cols, p):
    pos, neg = counts.row_trend_masks(np.asarray(x, np.float32), list(cols), p.neg_trends,
                                      p.ratio_num, p.ratio_den)
    return set(np.flatnonzero(pos)), set(np.flatnonzero(neg))


# Hand-worked example (our own, from the definition in Sec. 2.3):
#   r0 = [1,2,3,4]  r1 = [4,3,2,1]  r2 = [1,3,3,2], individual I = (0,1,2).
#   r0: pairs (1<2),(2<3) -> 2 increases; r1: 2 decreases; r2: (1<3) increase, (3=3) tie.
#   exact: pos {r0}, neg {r1}; ratio 1/2 -> t = ceil(1/2 * 2) = 1: pos {r0, r2}, neg {r1}.
#   reverse(I) = (2,1,0): r1 read as [2,3,4] increases -> pos {r1} = neg(I).
HAND = np.array([[1, 2, 3, 4], [4, 3, 2, 1], [1, 3, 3, 2]], dtype=np.float32)


def test_hand_example_exact():
    assert masks(HAND, (0, 1, 2), P()) == ({0}, {1})


def test_hand_example_half_ratio():
    assert masks(HAND, (0, 1, 2), P(ratio_num=1, ratio_den=2)) == ({0, 2}, {1})


def test_hand_example_reverse():
    pos_rev, _ = masks(HAND, (2, 1, 0), P())
    assert pos_rev == {1}


def test_hand_example_counts_and_fitness():
    p = P(min_rows=2, col_cap=10)
    rp, rn, ra, f = counts.eval_individual(HAND, [0, 1, 2], p)
    assert (rp, rn, ra) == (1, 1, 2)
    assert f == 2 * 2 ** 3
    p.min_rows = 3
    assert counts.eval_individual(HAND, [0, 1, 2], p)[3] == 0


def test_negative_trends_switch():
    assert masks(HAND, (0, 1, 2), P(neg_trends=0)) == ({0}, set())


@pytest.mark.parametrize("num,den", [(85, 100), (1, 2), (2, 3), (1, 1), (1, 100), (99, 100)])
def test_threshold_is_ceiling(num, den):
    for L in range(2, 65):
        assert counts.threshold(L, num, den) == math.ceil(Fraction(num, den) * (L - 1))


def test_threshold_values():
    assert counts.threshold(2, 85, 100) == 1
    assert counts.threshold(7, 85, 100) == 6      # 0.85 * 6 = 5.1 -> 6
    assert counts.threshold(8, 85, 100) == 6      # 5.95 -> 6
    assert counts.threshold(21, 85, 100) == 17    # 17.0 exactly
    assert counts.threshold(64, 85, 100) == 54    # 53.55 -> 54
    assert counts.threshold(64, 1, 1) == 63


def per_row_loop(x, cols, neg, num, den):
    """Independent formulation: a Python loop over rows and pairs, threshold by Fraction."""
    rp = rn = ra = 0
    need = Fraction(num, den) * (len(cols) - 1)
    for row in x.tolist():
        v = [row[c] for c in cols]
        inc = sum(1 for a, b in zip(v, v[1:]) if b > a)
        dec = sum(1 for a, b in zip(v, v[1:]) if b < a)
        po = inc >= need
        ne = bool(neg) and dec >= need
        rp += po
        rn += ne
        ra += po or ne
    return rp, rn, ra


def test_counts_match_row_loop_on_ties_and_zeros():
    g = np.random.default_rng(1)
    x = g.integers(-3, 4, size=(97, 9)).astype(np.float32) * 0.5
    x[::7, 2] = -0.0
    x[::5, 3] = 0.0
    x[::11, 4] = np.float32(1e-45)      # denormal
    x[::13, 5] = np.float32(-1e-45)
    for num, den in [(1, 1), (85, 100), (1, 2)]:
        p = P(ratio_num=num, ratio_den=den)
        for L in range(2, 9):
            for _ in range(5):
                cols = list(g.choice(9, size=L, replace=False))
                assert counts.eval_individual(x, cols, p)[:3] == per_row_loop(x, cols, 1, num, den)


def test_signed_zero_is_a_tie():
    x = np.array([[0.0, -0.0], [-0.0, 0.0], [-1.0, 0.0]], dtype=np.float32)
    assert masks(x, (0, 1), P()) == ({2}, set())


def test_reversal_symmetry():
    g = np.random.default_rng(2)
    x = g.standard_normal((300, 12)).astype(np.float32)
    x[:, 5] = x[:, 6]                    # ties
    for num, den in [(1, 1), (85, 100), (3, 5)]:
        p = P(ratio_num=num, ratio_den=den)
        for L in range(2, 12):
            cols = list(g.choice(12, size=L, replace=False))
            rp, rn, _, _ = counts.eval_individual(x, cols, p)
            rp_rev, rn_rev, _, _ = counts.eval_individual(x, cols[::-1], p)
            assert rp_rev == rn and rn_rev == rp


def test_exact_never_exceeds_approx_and_shrinks_on_append():
    g = np.random.default_rng(3)
    x = g.standard_normal((400, 10)).astype(np.float32)
    for _ in range(40):
        L = int(g.integers(2, 10))
        cols = list(g.choice(10, size=L, replace=False))
        ex = counts.eval_individual(x, cols, P())
        ap = counts.eval_individual(x, cols, P(ratio_num=85, ratio_den=100))
        assert all(e <= a for e, a in zip(ex[:3], ap[:3]))
        extra = [c for c in range(10) if c not in cols][0]
        ex2 = counts.eval_individual(x, cols + [extra], P())
        assert all(e2 <= e for e2, e in zip(ex2[:3], ex[:3]))


def test_ratio_just_below_one_equals_exact():
    g = np.random.default_rng(4)
    x = g.standard_normal((200, 64)).astype(np.float32)
    for L in (2, 17, 64):
        cols = list(g.choice(64, size=L, replace=False))
        assert counts.eval_individual(x, cols, P(ratio_num=99, ratio_den=100)) == \
            counts.eval_individual(x, cols, P())


def test_length_two_approx_equals_exact():
    g = np.random.default_rng(5)
    x = g.standard_normal((200, 6)).astype(np.float32)
    for a, b in itertools.permutations(range(6), 2):
        assert counts.eval_individual(x, [a, b], P(ratio_num=1, ratio_den=100)) == \
            counts.eval_individual(x, [a, b], P())


def test_constant_matrix_has_no_trend():
    x = np.full((50, 6), 3.25, dtype=np.float32)
    for num, den in [(1, 1), (1, 2), (1, 100)]:
        assert counts.eval_individual(x, [0, 3, 1, 5], P(ratio_num=num, ratio_den=den))[:3] == (0, 0, 0)


def test_brute_force_recovers_planted_order():
    """Tiny matrix (8 x 6): 5 rows follow column order (4, 1, 3) increasing; the planted order is
    the unique argmax of rows_pos among all length-3 sequences, and with negative trends on, its
    reverse ties it on rows_any; the reverse's rows are its negative rows."""
    g = np.random.default_rng(6)
    x = g.standard_normal((8, 6)).astype(np.float32)
    order = (4, 1, 3)
    for r in range(5):
        x[r, list(order)] = np.sort(g.standard_normal(3)).astype(np.float32) + np.array([0, 2, 4], np.float32)
    p = P(neg_trends=0)
    best = {}
    for L in (2, 3, 4):
        for seq in itertools.permutations(range(6), L):
            rp = counts.eval_individual(x, list(seq), p)[0]
            best.setdefault(L, []).append((rp, seq))
    scores3 = sorted(best[3], reverse=True)
    assert scores3[0][1] == order and scores3[0][0] >= 5 and scores3[1][0] < scores3[0][0]
    pn = P(neg_trends=1)
    fwd = counts.eval_individual(x, list(order), pn)
    rev = counts.eval_individual(x, list(order[::-1]), pn)
    assert fwd[2] == rev[2] and rev[1] == fwd[0]


def test_planted_rows_are_recovered():
    """Every planted row without a noise-induced violation of its order is counted."""
    w = synth.WORKLOADS["tiny"]
    x, truth, _, _ = synth.workload_inputs(w)
    p = P(neg_trends=1)
    for k, (ridx, order, sign) in enumerate(truth):
        seq = list(order) if sign > 0 else list(order[::-1])
        vals = x[np.ix_(ridx, seq)]
        clean = int((np.diff(vals, axis=1) > 0).all(axis=1).sum())
        rp, rn, ra, _ = counts.eval_individual(x, seq, p)
        assert rp >= clean > 0
        if k == len(truth) - 1:          # the last planted bicluster is never overwritten
            assert clean >= len(ridx) - 2


def test_fitness_rule():
    assert counts.fitness(1, 5, 2, 10) == 0
    assert counts.fitness(2, 5, 2, 10) == 2 << 5
    assert counts.fitness(7, 40, 2, 10) == 7 << 10
    assert counts.fitness(7, 40, 2, 10, dead=True) == 0


def test_bitmap_definition_against_counts():
    """AND of the consecutive pair words reproduces the exact positive and negative row sets."""
    g = np.random.default_rng(7)
    x = g.integers(0, 4, size=(77, 7)).astype(np.float32)
    G = pair_bitmap(x)
    W = G.shape[2]
    for a in range(7):
        for b in range(7):
            if a != b:
                assert not (G[a, b] & G[b, a]).any()
    for _ in range(30):
        L = int(g.integers(2, 6))
        cols = list(g.choice(7, size=L, replace=False))
        acc_p = np.full(W, 0xFFFFFFFF, np.uint32)
        acc_n = np.full(W, 0xFFFFFFFF, np.uint32)
        for u, v in zip(cols, cols[1:]):
            acc_p &= G[u, v]
            acc_n &= G[v, u]
        popc = lambda a: sum(bin(int(w)).count("1") for w in a)
        rp, rn, _, _ = counts.eval_individual(x, cols, P())
        assert popc(acc_p) == rp and popc(acc_n) == rn


def test_bitmap_layout_hand_worked():
    """The word layout written out by hand: bit j of word w is row 32w + j, G[a][b] marks rows
    where column b is strictly greater than column a, ties (including -0 against +0) set no bit,
    subnormals compare by value, and rows past the end are 0.  40 rows, so the second word holds
    rows 32..39 only."""
    R = 40
    x = np.zeros((R, 3), np.float32)
    x[[0, 3, 31, 32, 39], 1] = 1.0          # column 1 above column 0 on these rows
    x[[1, 33], 1] = -1.0                    # and below it on these
    x[:, 2] = -0.0                          # -0 ties +0 everywhere ...
    x[5, 2] = np.float32(1e-45)             # ... except a positive subnormal on row 5
    x[34, 2] = -np.float32(1e-45)           # and a negative one on row 34
    G = pair_bitmap(x)
    assert G.shape == (3, 3, 2)
    assert [int(v) for v in G[0, 1]] == [0x80000009, 0x00000081]   # rows 0, 3, 31 | 32, 39
    assert [int(v) for v in G[1, 0]] == [0x00000002, 0x00000002]   # row 1 | row 33
    assert [int(v) for v in G[0, 2]] == [0x00000020, 0x00000000]   # row 5
    assert [int(v) for v in G[2, 0]] == [0x00000000, 0x00000004]   # row 34
    # column 1 against column 2: +1 is above every entry of column 2 and -1 below; a 0 of
    # column 1 ties -0, lies below the positive subnormal (row 5) and above the negative one
    # (row 34)
    assert [int(v) for v in G[2, 1]] == [0x80000009, 0x00000085]   # rows 0, 3, 31 | 32, 34, 39
    assert [int(v) for v in G[1, 2]] == [0x00000022, 0x00000002]   # rows 1, 5 | 33
    for a in range(3):
        assert not G[a, a].any()
    assert [int(v) for v in pair_words(x, 0, 1)] == [0x80000009, 0x00000081]


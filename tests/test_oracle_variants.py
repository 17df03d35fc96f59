"""Pins of the oracle's two trend variants (no GPU): ties that count for both directions
(non_strict) and counting against the last value that kept the trend (last_kept).

Hand-worked examples written from the definitions, a plain per-row loop, and the invariants the
definitions imply."""

import numpy as np
import pytest

from oracle import counts
from oracle.params import Params


def P(**kw):
    base = dict(neg_trends=1, ratio_num=1, ratio_den=1, min_rows=0, col_cap=10)
    base.update(kw)
    return Params(**base)


def masks(x, cols, p):
    pos, neg = counts.row_trend_masks(np.asarray(x, np.float32), list(cols), p.neg_trends,
                                      p.ratio_num, p.ratio_den, p.non_strict, p.last_kept)
    return set(np.flatnonzero(pos)), set(np.flatnonzero(neg))


# r0 = [1,2,3,4], r1 = [4,3,2,1], r2 = [1,3,3,2], individual (0,1,2).  With ties counting for both
# directions r2 reads (1 <= 3), (3 = 3): both pairs hold upwards, the first fails downwards.
HAND = np.array([[1, 2, 3, 4], [4, 3, 2, 1], [1, 3, 3, 2]], dtype=np.float32)


def test_non_strict_hand_example():
    assert masks(HAND, (0, 1, 2), P()) == ({0}, {1})
    assert masks(HAND, (0, 1, 2), P(non_strict=1)) == ({0, 2}, {1})


def test_non_strict_signed_zero_and_constant_rows():
    x = np.array([[0.0, -0.0], [-0.0, 0.0], [-1.0, 0.0], [2.0, 2.0]], dtype=np.float32)
    assert masks(x, (0, 1), P(non_strict=1)) == ({0, 1, 2, 3}, {0, 1, 3})


# Rows over columns (0,1,2,3), ratio 2/3 -> t = ceil(2/3 * 3) = 2 of the 3 steps:
#   A = [1,5,2,3]: consecutive ups (1<5),(2<3) = 2;  last kept: 5>1 (keep 5), 2, 3 below 5 = 1.
#   B = [4,1,3,2]: consecutive downs (4>1),(3>2) = 2; last kept: 1<4 (keep 1), 3, 2 above 1 = 1.
#   C = [1,3,2,4]: consecutive ups 2; last kept: 3>1 (keep 3), 2 skipped, 4>3 = 2.
LK = np.array([[1, 5, 2, 3], [4, 1, 3, 2], [1, 3, 2, 4]], dtype=np.float32)


def test_last_kept_hand_example():
    cols = (0, 1, 2, 3)
    assert masks(LK, cols, P(ratio_num=2, ratio_den=3)) == ({0, 2}, {1})
    assert masks(LK, cols, P(ratio_num=2, ratio_den=3, last_kept=1)) == ({2}, set())


def test_last_kept_with_ties():
    # [1,1,0,2] upwards with ties: 1>=1 (keep 1), 0 skipped, 2>=1 -> 2 of 3; strict: 2>1 -> 1.
    x = np.array([[1, 1, 0, 2]], dtype=np.float32)
    p = P(ratio_num=2, ratio_den=3, neg_trends=0, last_kept=1)
    assert masks(x, (0, 1, 2, 3), p) == (set(), set())
    p.non_strict = 1
    assert masks(x, (0, 1, 2, 3), p) == ({0}, set())


def per_row_loop(x, cols, non_strict, last_kept):
    """Counts (inc, dec) per row with a plain Python loop."""
    out = []
    for row in x:
        v = [float(row[c]) for c in cols]
        res = []
        for positive in (True, False):
            def holds(nxt, prev):
                if positive:
                    return nxt >= prev if non_strict else nxt > prev
                return nxt <= prev if non_strict else nxt < prev
            n = 0
            last = v[0]
            for k in range(1, len(v)):
                ref = last if last_kept else v[k - 1]
                if holds(v[k], ref):
                    n += 1
                    last = v[k]
            res.append(n)
        out.append(tuple(res))
    return out


@pytest.mark.parametrize("non_strict,last_kept", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_variants_match_row_loop(non_strict, last_kept):
    g = np.random.default_rng(3 + 2 * non_strict + last_kept)
    x = g.integers(-2, 3, size=(60, 10)).astype(np.float32)
    x[::7, 3] = -0.0
    for L in (2, 3, 5, 8, 10):
        cols = list(g.choice(10, size=L, replace=False))
        want = per_row_loop(x, cols, non_strict, last_kept)
        sub = x[:, cols]
        inc = counts.trend_count(sub, True, non_strict, last_kept)
        dec = counts.trend_count(sub, False, non_strict, last_kept)
        assert [(int(a), int(b)) for a, b in zip(inc, dec)] == want


def test_variant_invariants():
    g = np.random.default_rng(11)
    x = g.integers(0, 4, size=(400, 12)).astype(np.float32)
    for L in range(2, 13):
        cols = list(g.choice(12, size=L, replace=False))
        sub = x[:, cols]
        for positive in (True, False):
            for ns in (0, 1):
                cons = counts.trend_count(sub, positive, ns, 0)
                lk = counts.trend_count(sub, positive, ns, 1)
                # a step kept against the last kept value also holds against its predecessor
                # (the predecessor is the kept value or lies on the wrong side of it)
                assert (lk <= cons).all()
                # every step kept <=> every consecutive pair holds
                assert ((lk == L - 1) == (cons == L - 1)).all()
            strict = counts.trend_count(sub, positive, 0, 0)
            assert (counts.trend_count(sub, positive, 1, 0) >= strict).all()
        # with ties counting both ways, every pair holds in at least one direction
        up = counts.trend_count(sub, True, 1, 0)
        down = counts.trend_count(sub, False, 1, 0)
        assert (up + down >= L - 1).all()

"""Scripted-word pins of the oracle's variation operators and tournament (the readings of Sec.
2.3's strategies: one mutation chosen by the top two bits of a word, infeasible operators redrawn
at most 8 times and then a swap, new columns drawn at most 64 times; a tournament of T uniform
draws with ties to the lower slot; a one-point crossover when the word is below 2^30).

Each case feeds hand-chosen words and checks the chromosome worked out by hand from those
readings, so a wrong position, a dropped redraw or a swapped operand in the oracle fails here.
A uniform draw below(n) is the high word of w * n."""

from types import SimpleNamespace

import pytest

from oracle import ebic
from oracle.params import Params


class Script:
    """A word stream that returns the given words in order (and fails when they run out)."""

    def __init__(self, words):
        self.words = list(words)

    def next(self):
        return self.words.pop(0)

    def below(self, n):
        return (self.next() * n) >> 32


def w(k, n):
    """The smallest word with below(n) == k."""
    return -(-(k << 32) // n)


def op(k):
    """A word whose top two bits select operator k (0 insert, 1 delete, 2 substitute, 3 swap)."""
    return k << 30


def mutated(child, words, n_cols=10, max_len=6):
    s = Script(words)
    c = list(child)
    ebic.mutate(s, c, n_cols, max_len)
    assert s.words == [], "every scripted word is used, no more"
    return c


def test_word_helper():
    for n in (1, 2, 3, 7, 10, 64, 1000):
        for k in range(min(n, 9)):
            assert (w(k, n) * n) >> 32 == k


def test_insert_redraws_a_present_column():
    # position 1 of 4, column 5 is present, column 2 is free
    assert mutated([3, 5, 7], [op(0), w(1, 4), w(5, 10), w(2, 10)]) == [3, 2, 5, 7]


def test_delete():
    assert mutated([3, 5, 7], [op(1), w(2, 3)]) == [3, 5]


def test_delete_at_length_two_is_redrawn():
    # delete is infeasible at L = 2; the next word picks substitute: position 0, column 9
    assert mutated([3, 5], [op(1), op(2), w(0, 2), w(9, 10)]) == [9, 5]


def test_substitute_redraws_present_columns():
    assert mutated([3, 5, 7], [op(2), w(1, 3), w(5, 10), w(7, 10), w(4, 10)]) == [3, 4, 7]


def test_swap_positions():
    # p = 0, q = below(2) = 0 >= p -> q = 1
    assert mutated([3, 5, 7], [op(3), w(0, 3), w(0, 2)]) == [5, 3, 7]
    # p = 2, q = 0 < p
    assert mutated([3, 5, 7], [op(3), w(2, 3), w(0, 2)]) == [7, 5, 3]


def test_insert_at_max_len_and_substitute_with_every_column_used():
    # L = max_len = n_cols = 6: insert and substitute are infeasible; after 8 of them, a swap
    words = [op(0), op(2)] * 4 + [w(4, 6), w(1, 5)]
    assert mutated(list(range(6)), words, n_cols=6, max_len=6) == [0, 4, 2, 3, 1, 5]


def test_new_column_gives_up_after_64_draws():
    # n_cols = 3 and all 64 draws return column 0, which is present: the insert (position 0)
    # is infeasible, so is a delete at L = 2, and the swap follows
    words = [op(0), w(0, 3)] + [w(0, 3)] * 64 + [op(1), op(3), w(1, 2), w(0, 1)]
    assert mutated([0, 1], words, n_cols=3) == [1, 0]


def pop_state(fit, pen, pop=None):
    n = len(fit)
    return SimpleNamespace(pop=pop or [[0, 1]] * n, fit=list(fit), penalty=list(pen))


def test_tournament_ties_go_to_the_lower_slot():
    st = pop_state([8, 4, 8, 2], [1, 0, 1, 0])      # scores 4, 4, 4, 2
    assert ebic.tournament(Script([w(2, 4), w(1, 4), w(0, 4)]), st, 3) == 0
    assert ebic.tournament(Script([w(3, 4), w(2, 4)]), st, 2) == 2


def test_tournament_takes_the_best_penalised_score():
    st = pop_state([8, 4, 16, 2], [1, 0, 1, 0])     # scores 4, 4, 8, 2
    assert ebic.tournament(Script([w(3, 4), w(0, 4), w(2, 4)]), st, 3) == 2
    assert ebic.tournament(Script([w(1, 4)]), st, 1) == 1


def child_with(monkeypatch, st, words, **kw):
    s = Script(words)
    monkeypatch.setattr(ebic, "WordStream", lambda *a: s)
    p = Params(**dict(dict(tournament=1, max_len=6, seed=1), **kw))
    c = ebic.make_child(st, p, 10, 1, 0, 0)
    assert s.words == []
    return c


def test_crossover_child(monkeypatch):
    st = pop_state([1, 1, 1], [0, 0, 0], pop=[[0, 1, 2, 3], [4, 2, 5], [6, 7]])
    # parent 0; crossover (word 0 < 2^30) with parent 1; cut1 = 1 + 1 = 2 -> [0, 1];
    # cut2 = 1 + 0 = 1 -> [2, 5] (none already present); then delete position 3
    words = [w(0, 3), 0, w(1, 3), w(1, 3), w(0, 2), op(1), w(3, 4)]
    assert child_with(monkeypatch, st, words) == [0, 1, 2]


def test_crossover_drops_repeated_columns_and_cuts_to_max_len(monkeypatch):
    st = pop_state([1, 1], [0, 0], pop=[[0, 1, 2, 3, 4], [9, 8, 1, 7, 6, 5]])
    # cut1 = 1 + 3 = 4 -> [0, 1, 2, 3]; cut2 = 1 + 0 = 1 -> [8, 1, 7, 6, 5] minus 1 ->
    # [0, 1, 2, 3, 8, 7, 6, 5] cut to 6 -> [0, 1, 2, 3, 8, 7]; then swap positions 0 and 5
    words = [w(0, 2), 0, w(1, 2), w(3, 4), w(0, 5), op(3), w(0, 6), w(4, 5)]
    assert child_with(monkeypatch, st, words) == [7, 1, 2, 3, 8, 0]


def test_no_crossover_at_the_threshold_word(monkeypatch):
    st = pop_state([1, 1], [0, 0], pop=[[0, 1, 2], [4, 5, 6]])
    # the word 2^30 is not below 2^30: the child copies parent 1, then delete position 0
    words = [w(1, 2), 1 << 30, op(1), w(0, 3)]
    assert child_with(monkeypatch, st, words) == [5, 6]


def init_with(monkeypatch, words, n_cols=10, **kw):
    s = Script(words)
    monkeypatch.setattr(ebic, "WordStream", lambda *a: s)
    p = Params(**dict(dict(init_min_len=2, init_max_len=4, max_len=6, seed=1), **kw))
    c = ebic.init_individual(p, n_cols, 0)
    assert s.words == []
    return c


def test_initial_chromosome(monkeypatch):
    # length 2 + below(3) = 4; column 5, then 5 again (present, redrawn) -> 1, then 9, then 0
    words = [w(2, 3), w(5, 10), w(5, 10), w(1, 10), w(9, 10), w(0, 10)]
    assert init_with(monkeypatch, words) == [5, 1, 9, 0]


def test_initial_chromosome_ends_after_64_failed_draws(monkeypatch):
    # length 2 + below(2) = 3 with init_max_len = 3; column 0, then 64 draws of column 0: the
    # chromosome ends there (the third column is never drawn)
    words = [w(1, 2), w(0, 3)] + [w(0, 3)] * 64
    assert init_with(monkeypatch, words, n_cols=3, init_max_len=3) == [0]

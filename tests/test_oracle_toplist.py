"""Hand-worked pins of the oracle's top-rank-list update and duplicate rule (the readings of Sec.
2.3's top list and tabu list): candidates are taken by (fitness desc, key asc); a key already in
the list is skipped, so is a candidate ranking at position >= K; a candidate may share at most
overlap_num / overlap_den of *its own* columns with every better entry; once admitted, worse
entries sharing more than that fraction of *their* columns with it are evicted; the list is cut
to K.  Among live slots from `first` on, equal keys keep the lowest slot, each repeat being one
hit.  Every expected list below is worked out by hand from those rules."""

from oracle import ebic
from oracle.ebic import Entry
from oracle.params import Params


def E(cols, f, h):
    return Entry(tuple(cols), f, h, 0, 0, 0)


def keys(top):
    return [e.h for e in top]


P3 = Params(n_biclusters=3, elite=3, overlap_num=1, overlap_den=2)
P2 = Params(n_biclusters=2, elite=2, overlap_num=1, overlap_den=2)


def test_admission_order_overlap_and_capacity():
    A = E((0, 1, 2, 3), 100, 1)
    B = E((0, 1, 4, 5), 90, 2)   # shares 2 of its 4 columns with A: 2/4 <= 1/2, admitted
    C = E((0, 1, 2, 6), 80, 3)   # shares 3 of 4 with A: rejected
    D = E((7, 8), 70, 4)         # disjoint: admitted at position 2
    F = E((9, 10), 60, 5)        # would rank at position 3 = K: skipped
    assert keys(ebic.update_toplist([], [F, D, C, B, A], P3)) == [1, 2, 4]


def test_overlap_is_measured_on_the_candidates_own_columns():
    A = E((0, 1, 2, 3), 100, 1)
    small = E((0, 1), 95, 7)     # shares 2 of its own 2 columns with A: rejected
    assert keys(ebic.update_toplist([A], [small], P3)) == [1]
    # the same columns the other way round: A would share 2 of its 4 with `small`, and is kept
    # when it is the worse entry
    small_better = E((0, 1), 120, 7)
    assert keys(ebic.update_toplist([A], [small_better], P3)) == [7, 1]


def test_admission_evicts_worse_entries_it_overlaps():
    A = E((0, 1, 2, 3), 100, 1)
    D = E((7, 8), 70, 4)
    F = E((7, 8, 9), 80, 6)      # ranks at 1; D shares 2 of its 2 columns with F: evicted
    assert keys(ebic.update_toplist([A, D], [F], P3)) == [1, 6]


def test_eviction_happens_before_the_next_candidates_position():
    A = E((0, 1, 2, 3), 100, 1)
    D = E((7, 8), 70, 4)
    F = E((7, 8, 9), 80, 6)
    X = E((20, 21), 60, 8)       # after F evicts D the list holds 2 = K entries: X ranks at 2
    assert keys(ebic.update_toplist([A, D], [X, F], P2)) == [1, 6]
    # with K = 3, X takes the place D left
    assert keys(ebic.update_toplist([A, D], [X, F], P3)) == [1, 6, 8]


def test_equal_fitness_ranks_by_key_and_known_keys_are_skipped():
    G = E((0, 1), 50, 10)
    H = E((2, 3), 50, 9)
    assert keys(ebic.update_toplist([], [G, H], P2)) == [9, 10]
    # a candidate whose key is already listed is skipped, whatever else it carries
    assert keys(ebic.update_toplist([H], [E((4, 5), 99, 9)], P2)) == [9]


def test_a_better_candidate_pushes_the_last_entry_out():
    A = E((0, 1), 100, 1)
    B = E((2, 3), 90, 2)
    Z = E((4, 5), 95, 3)         # ranks at 1 of K = 2: B is cut
    assert keys(ebic.update_toplist([A, B], [Z], P2)) == [1, 3]


def test_duplicates_keep_the_lowest_live_slot():
    pop = [[0]] * 6
    hashes = [11, 22, 11, 33, 22, 11]
    dead = [False, False, False, True, False, False]
    hits = ebic.dedup(pop, dead, hashes, first=1)
    # slot 0 is an elite (before `first`): slot 2's key 11 is its first live occurrence from
    # slot 1 on; slot 4 repeats 22 (slot 1) and slot 5 repeats 11 (slot 2); slot 3 was dead
    assert dead == [False, False, False, True, True, True] and hits == 2

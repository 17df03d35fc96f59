"""Hand-worked pins of the oracle's tabu rule and step 6 (the readings of Sec. 2.3's tabu list and
Sec. 2.4 step 6): elites copy the top list; any other slot retries with attempt a + 1 while its
child's key is in the tabu list as it stood at the generation's start, each retry being a hit;
after max_attempts hits the slot is dead and keeps its last child; equal keys among the live
non-elite slots keep the lowest slot, each repeat a hit; a generation whose hits reach
tabu_hit_limit is not scored.  The children are scripted per (slot, attempt)."""

import numpy as np

from oracle import ebic
from oracle.ebic import Entry, State
from oracle.fnv import chromosome_hash, tabu_key
from oracle.params import Params


def key(cols):
    return tabu_key(chromosome_hash(list(cols)))


def scripted_state(monkeypatch, limit):
    x = np.random.default_rng(0).standard_normal((8, 10)).astype(np.float32)
    p = Params(pop_size=5, elite=1, n_biclusters=2, max_attempts=3, tabu_hit_limit=limit,
               max_len=6, init_max_len=4, seed=1)
    old = [[0, 1], [2, 3], [4, 5], [6, 7], [8, 9]]
    st = State(gen=4, pop=[list(c) for c in old], dead=[False] * 5,
               hashes=[key(c) for c in old], fit=[1] * 5, penalty=[0] * 5,
               top=[Entry((0, 1), 1, key((0, 1)), 0, 0, 0)], tabu={key(c) for c in old})
    children = {
        (1, 0): [2, 3], (1, 1): [1, 2],                    # one hit, then a new child
        (2, 0): [4, 5], (2, 1): [6, 7], (2, 2): [8, 9],    # three hits: dead, keeps [8, 9]
        (3, 0): [3, 4],                                    # new
        (4, 0): [3, 4],                                    # new to the tabu list, repeats slot 3
    }
    calls = []

    def make_child(st_, p_, n_cols, g, s, a):
        calls.append((g, s, a))
        return list(children[(s, a)])

    monkeypatch.setattr(ebic, "make_child", make_child)
    return x, p, st, calls


def test_retries_dead_slots_and_repeats(monkeypatch):
    x, p, st, calls = scripted_state(monkeypatch, limit=0)
    assert ebic.next_generation(x, st, p)
    assert calls == [(5, 1, 0), (5, 1, 1), (5, 2, 0), (5, 2, 1), (5, 2, 2), (5, 3, 0), (5, 4, 0)]
    assert st.pop == [[0, 1], [1, 2], [8, 9], [3, 4], [3, 4]]
    assert st.dead == [False, False, True, False, True]
    assert st.hits[-1] == 1 + 3 + 1 and st.gen == 5
    # every live slot's key is in the tabu list after scoring; the dead slot's child is not
    assert {key([1, 2]), key([3, 4])} <= st.tabu
    assert st.fit[2] == 0 and st.fit[4] == 0


def test_hit_limit_stops_before_scoring(monkeypatch):
    x, p, st, calls = scripted_state(monkeypatch, limit=5)
    before = [list(c) for c in st.pop]
    assert not ebic.next_generation(x, st, p)
    assert st.stopped and st.hits[-1] == 5
    assert st.pop == before and st.gen == 4
    assert key([1, 2]) not in st.tabu


def test_hit_limit_not_reached(monkeypatch):
    x, p, st, calls = scripted_state(monkeypatch, limit=6)
    assert ebic.next_generation(x, st, p) and not st.stopped and st.gen == 5

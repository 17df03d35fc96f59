"""Invariants of the oracle's generation loop (Sec. 2.4 steps 1-9, Sec. 2.3 strategies).

The fitness formula, top-list rule and operators are readings the paper does not fix ("parity
unpinned" by the paper); these tests pin what the readings imply: valid chromosomes, a sorted
top list that obeys the overlap rule, no non-elite individual scored twice, exact penalised
tournament comparisons, step-6 termination, and resume equal to an uninterrupted run."""

from fractions import Fraction

import numpy as np
import pytest

from oracle import ebic
from oracle.counts import eval_individual
from oracle.fnv import chromosome_hash, tabu_key
from oracle.params import Params, validate
from oracle.philox import WordStream
from paper_2105_01196_gb300 import synth


def tiny_params(**kw):
    base = dict(neg_trends=1, ratio_num=85, ratio_den=100, max_len=6, init_min_len=2,
                init_max_len=6, pop_size=64, elite=4, n_biclusters=4, tabu_hit_limit=0, seed=11)
    base.update(kw)
    return Params(**base)


@pytest.fixture(scope="module")
def tiny():
    x, truth, _, _ = synth.workload_inputs(synth.WORKLOADS["tiny"])
    return x


def check_population(st, p, n_cols):
    for cols in st.pop:
        assert len(set(cols)) == len(cols)
        assert all(0 <= c < n_cols for c in cols)
    for s, cols in enumerate(st.pop):
        if not st.dead[s]:
            assert 2 <= len(cols) <= p.max_len


def check_toplist(top, p):
    keys = [(-e.f, e.h) for e in top]
    assert keys == sorted(keys)
    assert len({e.h for e in top}) == len(top) <= p.n_biclusters
    for i, e in enumerate(top):
        assert e.f > 0
        for better in top[:i]:
            inter = len(set(e.cols) & set(better.cols))
            assert inter * p.overlap_den <= p.overlap_num * len(e.cols)


def test_beats_matches_rational_comparison():
    g = np.random.default_rng(0)
    for _ in range(3000):
        fa, fb = (int(v) for v in g.integers(0, 1 << 20, size=2))
        ua, ub = (int(v) for v in g.integers(0, 70, size=2))
        if g.random() < 0.2:
            fb, ub = fa << 3, ua + 3     # exact ties
        ia, ib = 1, 2
        sa, sb = Fraction(fa, 2 ** ua), Fraction(fb, 2 ** ub)
        assert ebic.beats(fa, ua, ia, fb, ub, ib) == (sa > sb or (sa == sb and ia < ib))


def test_mutation_keeps_chromosomes_valid():
    for s in range(300):
        child = list(range(0, 2 + s % 5))
        stream = WordStream(5, 1, s, 0)
        before = list(child)
        ebic.mutate(stream, child, 8, 6)
        assert len(set(child)) == len(child) and 2 <= len(child) <= 6
        assert all(0 <= c < 8 for c in child)
        assert child != before or len(before) == 2  # a swap of two columns always changes it


def test_init_is_deterministic_and_valid(tiny):
    p = tiny_params()
    a = [ebic.init_individual(p, 20, s) for s in range(64)]
    b = [ebic.init_individual(p, 20, s) for s in range(64)]
    assert a == b
    for cols in a:
        assert p.init_min_len <= len(cols) <= p.init_max_len and len(set(cols)) == len(cols)


def test_run_invariants(tiny):
    p = tiny_params()
    st = ebic.run(tiny, p, 30)
    assert st.gen == 30 and not st.stopped
    check_population(st, p, 20)
    check_toplist(st.top, p)
    for e in st.top:
        rp, rn, ra, f = eval_individual(tiny, list(e.cols), p)
        assert (rp, rn, ra, f) == (e.rows_pos, e.rows_neg, e.rows_any, e.f)
    # elites are the top list's first entries
    n_el = min(p.elite, len(st.top))
    assert st.hits and all(h >= 0 for h in st.hits)
    assert n_el > 0


def test_no_non_elite_individual_scored_twice(tiny):
    p = tiny_params(seed=3)
    st = ebic.initialise(tiny, p)
    scored = set(st.hashes[s] for s in range(p.pop_size) if not st.dead[s])
    for _ in range(15):
        tabu_before = set(st.tabu)
        n_el = min(p.elite, len(st.top))
        assert ebic.next_generation(tiny, st, p)
        fresh = [st.hashes[s] for s in range(n_el, p.pop_size) if not st.dead[s]]
        assert len(fresh) == len(set(fresh))
        assert not (set(fresh) & tabu_before)
        for s in range(p.pop_size):
            assert st.hashes[s] == tabu_key(chromosome_hash(st.pop[s]))
        scored |= set(fresh)
    assert scored <= st.tabu


def test_tabu_limit_stops_before_scoring(tiny):
    p = tiny_params(pop_size=16, max_len=3, init_max_len=3, tabu_hit_limit=4, seed=5)
    st = ebic.run(tiny, p, 200)
    assert st.stopped
    assert st.hits[-1] >= 4
    assert st.gen == len(st.hits) - 2          # the stopping generation was not scored
    assert all(h < 4 for h in st.hits[1:-1])


def test_resume_equals_uninterrupted(tiny):
    import copy
    p = tiny_params(seed=9)
    full = ebic.run(tiny, p, 12)
    half = ebic.run(tiny, p, 5)
    saved = copy.deepcopy(half)
    resumed = ebic.run(tiny, p, 7, saved)
    assert resumed.pop == full.pop and resumed.top == full.top
    assert resumed.tabu == full.tabu and resumed.hits == full.hits


def test_extract_matches_counts(tiny):
    p = tiny_params(seed=2)
    st = ebic.run(tiny, p, 5)
    masks = ebic.extract(tiny, st, p)
    for e, m in zip(st.top, masks):
        assert sum(bin(int(w)).count("1") for w in m) == e.rows_any


def test_search_finds_planted_bicluster():
    """On an easy planted matrix the search's best entry is the planted order (quality, not
    parity): 40 rows follow a 4-column order in a 160 x 10 N(0,1) matrix."""
    x, truth = synth.planted_matrix(160, 10, 1, (40, 40), (4, 4), seed=77, neg_fraction=0.0)
    p = Params(neg_trends=0, ratio_num=1, ratio_den=1, max_len=5, init_min_len=2, init_max_len=4,
               pop_size=48, elite=4, n_biclusters=4, tabu_hit_limit=0, seed=4)
    st = ebic.run(x, p, 40)
    ridx, order, sign = truth[0]
    assert tuple(int(c) for c in order) in {e.cols for e in st.top}


def test_validate_rejects_bad_parameters():
    with pytest.raises(ValueError):
        validate(Params(ratio_num=0), 20)
    with pytest.raises(ValueError):
        validate(Params(max_len=30), 20)
    with pytest.raises(ValueError):
        validate(Params(elite=11, n_biclusters=10), 100)
    validate(Params(), 100)

"""The EBIC generation loop, step by step (Sec. 2.4, steps 1-9; strategies of Sec. 2.3).

Steps as the paper lists them:
  1. initialise a population of random short chromosomes (vectors of column numbers);
  2-3. score every individual: count its trend-preserving rows, turn the counts into scores and
     update the top rank list;
  4. start a new population with the best individuals of the top rank list (elitism);
  5. replenish it with mutated chromosomes of the old population, selected by a tournament that
     penalises frequently used columns (crowding); children whose hash is already in the tabu
     list are rejected;
  6. count the tabu-list hits of this generation; when they reach the threshold, stop (go to 9);
  7. score the population and update the top rank list;
  8. the new population replaces the old one; back to 4;
  9. the top rank list's chromosomes are scored once more and their accepted rows are returned.

Readings where the paper is silent:
  * Random words come from the Philox stream (generation g, slot s, attempt a), see ``philox``.
  * Initialisation (g = 0): length = init_min_len + below(init_max_len - init_min_len + 1), then
    columns drawn uniformly, a column already present is redrawn (at most 64 draws per column;
    if all 64 hit, the chromosome ends there and is dead when shorter than 2).
  * Elitism: slots 0..E'-1 take the first E' = min(elite, |top list|) top-list entries.
  * Tournament: T candidates drawn uniformly from the previous population; the penalised score of
    candidate i is f_i * 2**(-U_i), U_i = sum over its columns c of u(c), u(c) = number of
    top-list entries containing c; compared exactly; equal scores go to the lower slot.
  * A child copies its tournament winner; with probability 1/4 (word < 2**30) it is instead the
    one-point crossover of the winner with a second tournament winner: prefix p1[:cut1] with
    cut1 = 1 + below(L1 - 1), then p2[cut2:] with cut2 = 1 + below(L2 - 1) minus columns already
    present, truncated to max_len (shorter than 2 -> the copy of p1).
  * Then exactly one mutation: the operator is the top two bits of a word (0 insert, 1 delete,
    2 substitute, 3 swap); an infeasible operator is redrawn from the next word, at most 8 tries,
    after which the swap is applied.  Insert: position below(L+1) then a new column; delete:
    position below(L); substitute: position below(L) then a new column; swap: p = below(L),
    q = below(L-1), q += 1 when q >= p.  A new column is drawn as in initialisation (64 draws;
    failing all makes the operator infeasible).
  * Tabu: the hash is FNV-1a 64 (``fnv``).  A child whose key is in the tabu list as it stood at
    the start of the generation is a hit; the slot retries with attempt a + 1, up to
    max_attempts; after the last hit the slot is dead (fitness 0, not scored).  Among the live
    non-elite slots of one generation equal keys keep the lowest slot; the others are dead and
    each counts as a hit.  After scoring, every live slot's key enters the tabu list.
  * Step 6 compares the hits of the current generation with tabu_hit_limit (when > 0); the
    generation that reaches it is not scored and the run ends with the previous top list.
  * Top rank list (K = n_biclusters entries, sorted by fitness descending then tabu key
    ascending): the scored live slots with f > 0 are taken in that order; one whose key is in the
    list is skipped; one that would rank at position pos >= K is skipped; otherwise it must not
    share more than overlap_num/overlap_den of its own columns with any better entry; when
    admitted, worse entries that now share more than that fraction of *their* columns with it are
    removed, and the list is cut to K.

Test infrastructure only (see the package docstring).
"""

from collections import Counter
from dataclasses import dataclass, field

import numpy as np

from .counts import check_matrix, fitness, row_trend_masks
from .fnv import chromosome_hash, tabu_key
from .params import validate
from .philox import WordStream

CROSSOVER_BELOW = 1 << 30
OP_TRIES = 8
FREE_DRAWS = 64


@dataclass
class Entry:
    cols: tuple
    f: int
    h: int
    rows_pos: int
    rows_neg: int
    rows_any: int


@dataclass
class State:
    gen: int = -1
    pop: list = field(default_factory=list)
    dead: list = field(default_factory=list)
    hashes: list = field(default_factory=list)
    fit: list = field(default_factory=list)
    rows: list = field(default_factory=list)
    penalty: list = field(default_factory=list)
    top: list = field(default_factory=list)
    tabu: set = field(default_factory=set)
    stopped: bool = False
    hits: list = field(default_factory=list)
    n_evaluated: int = 0


# ----------------------------------------------------------------------------- selection

def beats(fa, ua, ia, fb, ub, ib):
    """True when candidate a wins against b: fa * 2**-ua > fb * 2**-ub, ties to the lower slot."""
    lhs = fa << ub
    rhs = fb << ua
    return lhs > rhs or (lhs == rhs and ia < ib)


def tournament(stream, st, size):
    P = len(st.pop)
    best = None
    for _ in range(size):
        i = stream.below(P)
        if best is None or beats(st.fit[i], st.penalty[i], i, st.fit[best], st.penalty[best], best):
            best = i
    return best


# ----------------------------------------------------------------------------- variation

def draw_free(stream, n_cols, child):
    for _ in range(FREE_DRAWS):
        c = stream.below(n_cols)
        if c not in child:
            return c
    return None


def swap_op(stream, child):
    L = len(child)
    p = stream.below(L)
    q = stream.below(L - 1)
    if q >= p:
        q += 1
    child[p], child[q] = child[q], child[p]


def mutate(stream, child, n_cols, max_len):
    for _ in range(OP_TRIES):
        op = stream.next() >> 30
        L = len(child)
        if op == 0:
            if L >= max_len or L >= n_cols:
                continue
            pos = stream.below(L + 1)
            c = draw_free(stream, n_cols, child)
            if c is None:
                continue
            child.insert(pos, c)
            return
        if op == 1:
            if L <= 2:
                continue
            pos = stream.below(L)
            del child[pos]
            return
        if op == 2:
            if L >= n_cols:
                continue
            pos = stream.below(L)
            c = draw_free(stream, n_cols, child)
            if c is None:
                continue
            child[pos] = c
            return
        swap_op(stream, child)
        return
    swap_op(stream, child)


def make_child(st, p, n_cols, g, s, a):
    stream = WordStream(p.seed, g, s, a)
    p1 = tournament(stream, st, p.tournament)
    if stream.next() < CROSSOVER_BELOW:
        p2 = tournament(stream, st, p.tournament)
        A, B = st.pop[p1], st.pop[p2]
        cut1 = 1 + stream.below(len(A) - 1)
        cut2 = 1 + stream.below(len(B) - 1)
        head = list(A[:cut1])
        child = head + [c for c in B[cut2:] if c not in head]
        child = child[:p.max_len]
        if len(child) < 2:
            child = list(A)
    else:
        child = list(st.pop[p1])
    mutate(stream, child, n_cols, p.max_len)
    return child


def init_individual(p, n_cols, s):
    stream = WordStream(p.seed, 0, s, 0)
    L = p.init_min_len + stream.below(p.init_max_len - p.init_min_len + 1)
    child = []
    for _ in range(L):
        c = draw_free(stream, n_cols, child)
        if c is None:
            break
        child.append(c)
    return child


# ----------------------------------------------------------------------------- tabu and dedup

def dedup(pop, dead, hashes, first):
    """Equal keys among live slots >= first keep the lowest slot; returns the added hits."""
    seen = set()
    hits = 0
    for s in range(first, len(pop)):
        if dead[s]:
            continue
        if hashes[s] in seen:
            dead[s] = True
            hits += 1
        else:
            seen.add(hashes[s])
    return hits


# ----------------------------------------------------------------------------- top rank list

def overlap_ok(cols, better_cols, p):
    inter = len(set(cols) & set(better_cols))
    return inter * p.overlap_den <= p.overlap_num * len(cols)


def update_toplist(top, cands, p):
    K = p.n_biclusters
    for c in sorted(cands, key=lambda e: (-e.f, e.h)):
        if any(e.h == c.h for e in top):
            continue
        pos = sum(1 for e in top if e.f > c.f or (e.f == c.f and e.h < c.h))
        if pos >= K:
            continue
        if not all(overlap_ok(c.cols, e.cols, p) for e in top[:pos]):
            continue
        top = top[:pos] + [c] + [e for e in top[pos:] if overlap_ok(e.cols, c.cols, p)]
        top = top[:K]
    return top


# ----------------------------------------------------------------------------- scoring

def row_counts(x, cols, p):
    """(rows_pos, rows_neg, rows_any) of one chromosome."""
    pos_ok, neg_ok = row_trend_masks(x, cols, p.neg_trends, p.ratio_num, p.ratio_den,
                                     p.non_strict, p.last_kept)
    return int(pos_ok.sum()), int(neg_ok.sum()), int((pos_ok | neg_ok).sum())


def score(x, st, p, counts_map=None):
    """Steps 2-3 / 7: counts and fitness of every live slot, then top list, tabu list, penalty.

    counts_map, when given, replaces the serial loop of ``row_counts`` over the live slots'
    chromosomes (a list in slot order -> their count triples, in the same order); it lets a
    caller spread the independent per-individual counts over several processes."""
    P = len(st.pop)
    st.fit = [0] * P
    st.rows = [(0, 0, 0)] * P
    cands = []
    live = [s for s in range(P) if not st.dead[s]]
    chroms = [st.pop[s] for s in live]
    counted = ([row_counts(x, c, p) for c in chroms] if counts_map is None
               else list(counts_map(chroms)))
    for s, (rp, rn, ra) in zip(live, counted):
        cols = st.pop[s]
        st.rows[s] = (rp, rn, ra)
        st.fit[s] = fitness(ra, len(cols), p.min_rows, p.col_cap)
        st.n_evaluated += 1
        if st.fit[s] > 0:
            cands.append(Entry(tuple(cols), st.fit[s], st.hashes[s], rp, rn, ra))
    st.top = update_toplist(st.top, cands, p)
    for s in range(P):
        if not st.dead[s]:
            st.tabu.add(st.hashes[s])
    use = Counter(c for e in st.top for c in e.cols)
    st.penalty = [sum(use[c] for c in st.pop[s]) for s in range(P)]


# ----------------------------------------------------------------------------- the loop

def initialise(x, p, counts_map=None):
    x = check_matrix(x)
    validate(p, x.shape[1])
    st = State()
    P = p.pop_size
    st.pop = [init_individual(p, x.shape[1], s) for s in range(P)]
    st.dead = [len(c) < 2 for c in st.pop]
    st.hashes = [tabu_key(chromosome_hash(c)) for c in st.pop]
    st.hits.append(dedup(st.pop, st.dead, st.hashes, 0))
    score(x, st, p, counts_map)
    st.gen = 0
    return st


def next_generation(x, st, p, counts_map=None):
    """Steps 4-8 for generation st.gen + 1; returns False when step 6 stopped the run."""
    n_cols = x.shape[1]
    g = st.gen + 1
    P = p.pop_size
    n_elite = min(p.elite, len(st.top))
    pop, dead, hashes = [], [], []
    hits = 0
    for s in range(P):
        if s < n_elite:
            pop.append(list(st.top[s].cols))
            dead.append(False)
            hashes.append(st.top[s].h)
            continue
        for a in range(p.max_attempts):
            child = make_child(st, p, n_cols, g, s, a)
            h = tabu_key(chromosome_hash(child))
            if h not in st.tabu:
                break
            hits += 1
        else:
            pop.append(child)
            dead.append(True)
            hashes.append(h)
            continue
        pop.append(child)
        dead.append(False)
        hashes.append(h)
    hits += dedup(pop, dead, hashes, n_elite)
    st.hits.append(hits)
    if p.tabu_hit_limit > 0 and hits >= p.tabu_hit_limit:
        st.stopped = True
        return False
    st.pop, st.dead, st.hashes = pop, dead, hashes
    score(x, st, p, counts_map)
    st.gen = g
    return True


def run(x, p, n_gen, st=None, counts_map=None):
    """Initialise when ``st`` is None, then run up to n_gen generations (fewer if step 6 stops).
    counts_map: see ``score``."""
    x = check_matrix(x)
    if st is None:
        st = initialise(x, p, counts_map)
    for _ in range(n_gen):
        if st.stopped or not next_generation(x, st, p, counts_map):
            break
    return st


def extract(x, st, p):
    """Step 9: row masks (uint32 words, bit j of word w = row 32w + j) of the top-list entries."""
    x = check_matrix(x)
    R = x.shape[0]
    W = (R + 31) // 32
    masks = np.zeros((len(st.top), W), dtype=np.uint32)
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    for k, e in enumerate(st.top):
        pos_ok, neg_ok = row_trend_masks(x, list(e.cols), p.neg_trends, p.ratio_num, p.ratio_den,
                                         p.non_strict, p.last_kept)
        bits = np.zeros(W * 32, dtype=np.uint64)
        bits[:R] = pos_ok | neg_ok
        masks[k] = (bits.reshape(W, 32) * weights).sum(axis=1).astype(np.uint32)
    return masks

"""GPU parity of the device generation loop with the oracle's step-by-step EBIC (Sec. 2.4 steps
1-9), through the C ABI.  Bar: identical populations, dead flags, fitness, top lists (columns,
fitness, keys, row counts), tabu-hit counts, stop generation and extracted row masks."""

import copy

import numpy as np
import pytest

from oracle import ebic as oebic
from oracle.fnv import chromosome_hash, tabu_key
from oracle.params import Params as OParams
from paper_2105_01196_gb300 import synth

pytestmark = pytest.mark.gpu

OKEYS = [f for f in OParams.__dataclass_fields__]


@pytest.fixture(scope="module")
def ebic():
    from paper_2105_01196_gb300 import ebic as e
    return e


def both_params(ebic, **kw):
    base = dict(neg_trends=1, ratio_num=85, ratio_den=100, max_len=6, init_min_len=2,
                init_max_len=6, pop_size=64, elite=4, n_biclusters=4, tabu_hit_limit=0, seed=11,
                min_rows=2, col_cap=10, overlap_num=1, overlap_den=2, tournament=4,
                max_attempts=4)
    base.update(kw)
    gp = ebic.Params.make(**base)
    op = OParams(**{k: v for k, v in base.items() if k in OKEYS})
    return gp, op


def assert_same_state(ctx, st, gp):
    top = ctx.toplist()
    assert len(top) == len(st.top)
    for g_e, o_e in zip(top, st.top):
        assert g_e["cols"] == tuple(o_e.cols)
        assert (g_e["f"], g_e["h"]) == (o_e.f, o_e.h)
        assert (g_e["rows_pos"], g_e["rows_neg"], g_e["rows_any"]) == \
            (o_e.rows_pos, o_e.rows_neg, o_e.rows_any)
        assert g_e["h"] == tabu_key(chromosome_hash(g_e["cols"]))
    cols, lens, dead, fit = ctx.population(gp.pop_size)
    for s in range(gp.pop_size):
        assert int(lens[s]) == len(st.pop[s]), f"slot {s}"
        assert list(cols[s, :lens[s]]) == list(st.pop[s]), f"slot {s}"
        assert bool(dead[s]) == st.dead[s], f"slot {s}"
        assert int(fit[s]) == st.fit[s], f"slot {s}"


def tiny_matrix():
    x, _, _, _ = synth.workload_inputs(synth.WORKLOADS["tiny"])
    return x


@pytest.mark.parametrize("mode,use_graph,ns,lk", [(1, 1, 0, 0), (2, 1, 0, 0), (2, 0, 0, 0),
                                                  (4, 1, 0, 0), (1, 1, 1, 1), (2, 1, 1, 0),
                                                  (0, 1, 0, 1)])
def test_generation_by_generation(ebic, mode, use_graph, ns, lk):
    x = tiny_matrix()
    gp, op = both_params(ebic, mode=mode, use_graph=use_graph, non_strict=ns, last_kept=lk)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        rep = ctx.run_generations(gp, 0)
        st = oebic.initialise(x, op)
        assert rep.gens_done == 0 and rep.n_evaluated == st.n_evaluated
        assert_same_state(ctx, st, gp)
        for g in range(1, 13):
            rep = ctx.run_generations(gp, 1)
            assert oebic.next_generation(x, st, op)
            assert rep.gens_done == g == st.gen
            assert rep.last_hits == st.hits[-1]
            assert rep.n_evaluated == st.n_evaluated
            assert_same_state(ctx, st, gp)


def test_long_run_and_extraction(ebic):
    x = tiny_matrix()
    gp, op = both_params(ebic, neg_trends=0, ratio_num=1, ratio_den=1, seed=3)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        rep = ctx.run_generations(gp, 60)
        st = oebic.run(x, op, 60)
        assert rep.gens_done == 60 and not rep.stopped
        assert rep.n_evaluated == st.n_evaluated
        assert_same_state(ctx, st, gp)
        masks = ctx.extract_biclusters(x.shape[0])
        want = oebic.extract(x, st, op)
        assert np.array_equal(masks[:, :want.shape[1]], want)
        assert not masks[:, want.shape[1]:].any()


def test_tabu_limit_stop(ebic):
    x = tiny_matrix()
    gp, op = both_params(ebic, pop_size=16, max_len=3, init_max_len=3, tabu_hit_limit=4, seed=5,
                         elite=2, n_biclusters=2)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        rep = ctx.run_generations(gp, 200)
        st = oebic.run(x, op, 200)
        assert st.stopped and rep.stopped == 1
        assert rep.gens_done == st.gen and rep.last_hits == st.hits[-1]
        assert_same_state(ctx, st, gp)
        rep2 = ctx.run_generations(gp, 5)           # a stopped run stays stopped
        assert rep2.gens_done == rep.gens_done


def test_checkpoint_resume(ebic):
    x = tiny_matrix()
    gp, op = both_params(ebic, seed=9)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        ctx.run_generations(gp, 5)
        blob = ctx.save_state()
        full = ctx.run_generations(gp, 7)
        top_full = ctx.toplist()
        pop_full = ctx.population(gp.pop_size)
    with ebic.Context(0) as ctx2:
        ctx2.load_matrix(x)
        ctx2.load_state(gp, blob)
        rep = ctx2.run_generations(gp, 7)
        assert rep.gens_done == full.gens_done == 12
        assert ctx2.toplist() == top_full
        for a, b in zip(ctx2.population(gp.pop_size), pop_full):
            assert np.array_equal(a, b)
    st = oebic.run(x, op, 12)
    assert [e["cols"] for e in top_full] == [tuple(e.cols) for e in st.top]


def test_default_workload_generations(ebic):
    """The default workload (10,000 x 100, P = 800, lengths 2-20, ratio 0.85, negative trends)
    for 20 generations against the oracle."""
    w = synth.WORKLOADS["default"]
    x, _, _, _ = synth.workload_inputs(w)
    gp, op = both_params(ebic, max_len=20, init_min_len=2, init_max_len=20, pop_size=800,
                         elite=10, n_biclusters=10, seed=w.seed)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        rep = ctx.run_generations(gp, 20)
        st = oebic.run(x, op, 20)
        assert rep.gens_done == st.gen == 20
        assert rep.n_evaluated == st.n_evaluated
        assert_same_state(ctx, st, gp)


@pytest.mark.parametrize("ns,ipw", [(0, 0), (1, 0), (0, 3), (1, 4)])
def test_generations_over_a_bitmap_larger_than_l2(ebic, ns, ipw):
    """The generation loop over a 243 MB pair bitmap (larger than the device's L2, so the bitmap
    kernel stages its pair words in shared memory) on a tie-heavy matrix, with ties counting for
    both directions or not, one individual per work item or groups of 3 or 4: generation by
    generation, then sixteen generations in one graph replay, against the oracle."""
    g = np.random.default_rng(21 + ns)
    x = g.integers(-3, 4, size=(4500, 650)).astype(np.float32)
    gp, op = both_params(ebic, mode=2, non_strict=ns, max_len=20, init_max_len=20, pop_size=96,
                         elite=6, n_biclusters=6, seed=23)
    gp.ipw = ipw                                    # (individuals per staged work item)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        ctx.run_generations(gp, 0)
        st = oebic.initialise(x, op)
        assert_same_state(ctx, st, gp)
        for gen in range(1, 4):
            rep = ctx.run_generations(gp, 1)
            assert oebic.next_generation(x, st, op)
            assert rep.gens_done == gen == st.gen
            assert rep.n_evaluated == st.n_evaluated
            assert_same_state(ctx, st, gp)
        rep = ctx.run_generations(gp, 16)
        for _ in range(16):
            assert oebic.next_generation(x, st, op)
        assert rep.gens_done == st.gen == 19
        assert rep.n_evaluated == st.n_evaluated
        assert_same_state(ctx, st, gp)


def test_run_parameter_errors(ebic):
    x = tiny_matrix()
    with ebic.Context(0) as ctx:
        with pytest.raises(ebic.EbicError):
            ctx.run_generations(ebic.Params.make(), 1)        # no matrix
        ctx.load_matrix(x)
        for bad in (dict(max_len=30), dict(elite=20, n_biclusters=10), dict(pop_size=1),
                    dict(tournament=0), dict(overlap_den=0), dict(mode=3)):
            gp, _ = both_params(ebic, **bad)
            with pytest.raises(ebic.EbicError) as e:
                ctx.run_generations(gp, 1)
            assert e.value.code == ebic.EBIC_EINVAL


@pytest.mark.parametrize("mode", [1, 2])
def test_same_shape_reload_starts_a_fresh_run(ebic, mode):
    """Loading a matrix of the same shape keeps the loop's buffers and graphs but starts a new run:
    each run equals the oracle's run on its own matrix, and nothing of the previous run is left."""
    x1 = tiny_matrix()
    x2, _ = synth.planted_matrix(x1.shape[0], x1.shape[1], 2, (30, 30), (5, 5), seed=99,
                                 neg_fraction=0.5)
    gp, op = both_params(ebic, mode=mode)
    with ebic.Context(0) as ctx:
        for x in (x1, x2, x1):
            ctx.load_matrix(x)
            with pytest.raises(ebic.EbicError) as e:
                ctx.toplist()                        # no run on this matrix yet
            assert e.value.code == ebic.EBIC_ESTATE
            rep = ctx.run_generations(gp, 8)
            st = oebic.run(x, op, 8)
            assert rep.gens_done == st.gen == 8
            assert rep.n_evaluated == st.n_evaluated
            assert_same_state(ctx, st, gp)


@pytest.mark.parametrize("tournament,max_attempts", [(1, 1), (3, 2), (6, 5), (8, 16)])
def test_tournament_and_attempt_shapes(ebic, tournament, max_attempts):
    """Tournament sizes on both sides of the paired-load path (T <= 4) and attempt counts that
    give 1, 2, 8 and 16 warps per slot, generation by generation against the oracle."""
    x = tiny_matrix()
    gp, op = both_params(ebic, mode=2, tournament=tournament, max_attempts=max_attempts, seed=21)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        ctx.run_generations(gp, 0)
        st = oebic.initialise(x, op)
        for g in range(1, 7):
            rep = ctx.run_generations(gp, 1)
            assert oebic.next_generation(x, st, op)
            assert rep.gens_done == g and rep.last_hits == st.hits[-1]
            assert_same_state(ctx, st, gp)


def test_large_population_multi_block_finish(ebic):
    """A population large enough for several k_finish blocks (their hand-over to the last block)
    and a candidate count past one warp, against the oracle."""
    x = tiny_matrix()
    gp, op = both_params(ebic, mode=1, pop_size=3000, elite=8, n_biclusters=8, seed=17)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        rep = ctx.run_generations(gp, 4)
        st = oebic.run(x, op, 4)
        assert rep.gens_done == st.gen == 4
        assert rep.n_evaluated == st.n_evaluated
        assert_same_state(ctx, st, gp)


def long_matrix(seed, ties):
    """700 x 128 with three planted trend biclusters of 40-64 columns, continuous values or, with
    ties, values rounded to integers and every third row constant."""
    x, _ = synth.planted_matrix(700, 128, 3, (80, 150), (40, 64), seed=seed, neg_fraction=0.34)
    if ties:
        x = np.round(x).astype(np.float32)
        x[::3] = 1.0
    return x


@pytest.mark.parametrize("mode,use_graph,ns,ratio,cap,init_lo", [
    (2, 1, 0, (1, 3), 16, 40), (1, 1, 0, (1, 3), 16, 2), (2, 0, 0, (1, 2), 16, 40),
    (1, 0, 1, (1, 2), 16, 40), (2, 1, 1, (1, 2), 16, 2), (4, 1, 0, (1, 3), 16, 40),
    (0, 1, 0, (1, 2), 16, 2), (1, 1, 0, (1, 1), 10, 40)])
def test_long_chromosomes_generation_by_generation(ebic, mode, use_graph, ns, ratio, cap,
                                                   init_lo):
    """Chromosomes of up to 64 columns (the warp's second 32 lanes: copies, mutation shifts,
    crossover suffixes past lane 32, the duplicate and penalty sums over 64 columns, top-list
    entries of more than 32 columns) on a 128-column matrix: initial lengths 40-64 or 2-64;
    bitmap, direct, staged and AUTO forms; graph-replayed and eager loops; strict and
    ties-for-both pair tests.  Low ratios with the column exponent capped at 16 make long
    chromosomes score best, so the population stays above 32 columns; the exact ratio lets it
    shrink after the first generations.  Ten generations one by one, then sixteen in one call
    (one graph replay), each against the oracle."""
    x = long_matrix(31 + init_lo + ns, ties=bool(ns))
    gp, op = both_params(ebic, mode=mode, use_graph=use_graph, non_strict=ns,
                         ratio_num=ratio[0], ratio_den=ratio[1], col_cap=cap, max_len=64,
                         init_min_len=init_lo, init_max_len=64, pop_size=96, elite=6,
                         n_biclusters=6, seed=41 + mode)
    longest, top_longest = [], []
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        rep = ctx.run_generations(gp, 0)
        st = oebic.initialise(x, op)
        assert rep.n_evaluated == st.n_evaluated
        assert_same_state(ctx, st, gp)
        for g in range(1, 11):
            rep = ctx.run_generations(gp, 1)
            assert oebic.next_generation(x, st, op)
            assert rep.gens_done == g == st.gen
            assert rep.last_hits == st.hits[-1]
            assert rep.n_evaluated == st.n_evaluated
            assert_same_state(ctx, st, gp)
            longest.append(max(len(c) for c in st.pop))
            top_longest.append(max((len(e.cols) for e in st.top), default=0))
        rep = ctx.run_generations(gp, 16)
        for _ in range(16):
            assert oebic.next_generation(x, st, op)
        assert rep.gens_done == st.gen == 26
        assert rep.n_evaluated == st.n_evaluated
        assert_same_state(ctx, st, gp)
    assert longest[0] > 32
    if ratio != (1, 1):
        assert min(longest) > 32
        assert ns or max(top_longest) > 32


@pytest.mark.parametrize("attempts,max_len,pop", [(4, 3, 1300), (16, 3, 400), (4, 64, 1500),
                                                  (2, 3, 1300)])
def test_sequential_attempt_form(ebic, attempts, max_len, pop):
    """Populations whose attempt warps exceed what the GPU holds at once (P x attempts rounded
    to a power of two > 152 SMs x 32 warps) run one warp per slot with the attempts in turn; two
    or three columns of a 20-column matrix make tabu hits and retries frequent, 64 columns of
    the 128-column matrix exercise the long paths.  (2 attempts x 1,300 slots stays in the
    one-block-per-slot form: the boundary from the other side.)  Generation by generation
    against the oracle."""
    x = tiny_matrix() if max_len == 3 else long_matrix(77, ties=False)
    kw = dict(init_max_len=3) if max_len == 3 else dict(init_min_len=40, init_max_len=64,
                                                         ratio_num=1, ratio_den=3, col_cap=16)
    gp, op = both_params(ebic, mode=2, max_attempts=attempts, max_len=max_len, pop_size=pop,
                         elite=6, n_biclusters=6, seed=29, **kw)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        ctx.run_generations(gp, 0)
        st = oebic.initialise(x, op)
        hits = 0
        for g in range(1, 7):
            rep = ctx.run_generations(gp, 1)
            assert oebic.next_generation(x, st, op)
            assert rep.gens_done == g and rep.last_hits == st.hits[-1]
            assert rep.n_evaluated == st.n_evaluated
            assert_same_state(ctx, st, gp)
            hits += st.hits[-1]
    assert max_len == 64 or hits > pop // 10


@pytest.mark.parametrize("fuse,neg,ns,ratio,pop,attempts,long_", [
    (63, 1, 0, (85, 100), 64, 4, False), (1, 1, 1, (85, 100), 64, 4, False),
    (2, 0, 0, (1, 2), 1300, 4, False), (63, 1, 1, (85, 100), 1300, 4, False),
    (63, 0, 0, (1, 1), 96, 4, True), (63, 1, 1, (1, 1), 1300, 4, True),
    (-1, 1, 0, (85, 100), 64, 4, False)])
def test_evaluation_inside_the_evolve_kernel(ebic, fuse, neg, ns, ratio, pop, attempts, long_):
    """Children whose pair test is exact (ceil(ratio x pairs) = pairs) and that have at most
    fuse_pairs pairs are evaluated by the warp that built them, inside the evolve kernel (one
    block per slot for 64 and 96 slots, a warp per slot for 1,300), the rest by the evaluation
    launch over the list of slots left to it; -1 turns it off.  Ratio 1 with chromosomes of up to
    64 columns puts pairs 32-62 in the fused path.  Generation by generation, then sixteen in one
    graph replay, against the oracle, with the number of fused evaluations checked."""
    x = long_matrix(53, ties=bool(ns)) if long_ else tiny_matrix()
    kw = (dict(max_len=64, init_min_len=40, init_max_len=64, col_cap=16) if long_ else {})
    gp, op = both_params(ebic, mode=2, neg_trends=neg, non_strict=ns, ratio_num=ratio[0],
                         ratio_den=ratio[1], pop_size=pop, max_attempts=attempts, elite=6,
                         n_biclusters=6, seed=61 + pop, **kw)
    gp.fuse_pairs = fuse
    fused = 0
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        rep = ctx.run_generations(gp, 0)
        st = oebic.initialise(x, op)
        assert rep.n_fused == 0                      # (the initial population has no evolve step)
        assert_same_state(ctx, st, gp)
        for g in range(1, 6):
            rep = ctx.run_generations(gp, 1)
            assert oebic.next_generation(x, st, op)
            assert rep.gens_done == g == st.gen
            assert rep.n_evaluated == st.n_evaluated
            assert_same_state(ctx, st, gp)
        rep = ctx.run_generations(gp, 16)
        for _ in range(16):
            assert oebic.next_generation(x, st, op)
        assert rep.gens_done == st.gen == 21
        assert rep.n_evaluated == st.n_evaluated
        assert_same_state(ctx, st, gp)
        fused = rep.n_fused
    if fuse < 0:
        assert rep.fuse_pairs == 0 and fused == 0 and rep.n_table == 0
    else:
        # (one-pair children are scored from the build's pair counts: 128 columns or fewer)
        assert rep.fuse_pairs == fuse and 0 < fused < rep.n_evaluated
        assert 0 <= rep.n_table <= fused and (long_ or rep.n_table > 0)

"""The autotuner's choices never change results: after tuning, EBIC_MODE_AUTO evaluations and
generations equal the oracle's."""

import numpy as np
import pytest

from oracle import counts as ocounts
from oracle import ebic as oebic
from oracle.params import Params as OParams
from paper_2105_01196_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sweeps", [1, 101])
def test_autotune_then_auto_matches_oracle(sweeps):
    from paper_2105_01196_gb300 import ebic
    w = synth.WORKLOADS["default"]
    x, _, ci, off = synth.workload_inputs(w)
    p = ebic.Params.make(neg_trends=1, ratio_num=85, ratio_den=100, mode=ebic.MODE_AUTO)
    op = OParams(neg_trends=1, ratio_num=85, ratio_den=100, min_rows=p.min_rows, col_cap=p.col_cap)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        rep = ctx.autotune(ci, off, p, sweeps)
        assert rep["mode"] in (ebic.MODE_DIRECT, ebic.MODE_BITMAP, ebic.MODE_STAGED)
        assert rep["direct_ms"] > 0 and rep["seg_direct"] >= 0 and rep["seg_bitmap"] >= 0
        assert rep["staged_ms"] > 0                  # 100 columns: the staged tiles fit
        # the loop's work-item size is measured when a run is expected (and p is a valid run)
        assert rep["seg_loop"] in (0, 1, 2, 4, 8, 16)
        assert sweeps > 2 or rep["seg_loop"] == 0
        got = ctx.eval_population(ci, off, p)
    want = ocounts.eval_population(x, ci, off, op)
    for g_, w_ in zip(got, want):
        assert np.array_equal(np.asarray(g_, np.int64), np.asarray(w_, np.int64))


def test_autotuned_generations_match_oracle():
    from paper_2105_01196_gb300 import ebic
    x, _, ci, off = synth.workload_inputs(synth.WORKLOADS["tiny"])
    base = dict(neg_trends=1, ratio_num=85, ratio_den=100, max_len=6, init_min_len=2,
                init_max_len=6, pop_size=64, elite=4, n_biclusters=4, tabu_hit_limit=0, seed=13)
    gp = ebic.Params.make(mode=ebic.MODE_AUTO, **base)
    op = OParams(**base)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        tune = ctx.autotune(ci, off, gp, 20)        # (its scratch runs of the loop are reset)
        rep = ctx.run_generations(gp, 20)
        top = ctx.toplist()
        pop = ctx.population(gp.pop_size)
        ctx.load_matrix(x)                          # a same-shape reload keeps the decisions
        rep2 = ctx.run_generations(gp, 20)
        assert ctx.toplist() == top
    st = oebic.run(x, op, 20)
    assert tune["seg_loop"] in (0, 1, 2, 4, 8, 16)
    # the loop's fusion limit is measured with the bitmap form only, and then used
    assert tune["fuse_loop"] in ((-1, 1, 2, 4, 8, 63) if tune["mode"] == ebic.MODE_BITMAP else (0,))
    if tune["mode"] == ebic.MODE_BITMAP:
        assert rep.fuse_pairs == max(tune["fuse_loop"], 0) == rep2.fuse_pairs
    assert rep.gens_done == rep2.gens_done == st.gen
    assert rep.n_evaluated == rep2.n_evaluated == st.n_evaluated
    assert [(e["cols"], e["f"]) for e in top] == [(tuple(e.cols), e.f) for e in st.top]
    assert [list(c[:n]) for c, n in zip(pop[0], pop[1])] == [list(c) for c in st.pop]


@pytest.mark.parametrize("R,C,seed", [(40000, 48, 3), (20000, 300, 4)])
def test_tuned_host_matrix_loads_in_segments(R, C, seed):
    """A host matrix of a shape the autotuner measured is copied in segments, each segment's
    keys, rank codes and bit planes built while the next one is copied, then (bitmap form) the
    pair words and counts in one launch: the load launches the rank-code kernel once per segment
    and the bitmap build once, and the results equal the oracle's (counts and fitness of a
    population; with the bitmap form, the pair words of a sample of pairs and the pair counts),
    with rows past the last segment boundary."""
    from oracle.bitmap import pair_words
    from paper_2105_01196_gb300 import ebic
    g = np.random.default_rng(seed)
    x = g.integers(-3, 4, size=(R, C)).astype(np.float32)
    x[g.random((R, C)) < 0.03] = -0.0
    lens = g.integers(2, 9, size=64)
    ci = np.concatenate([g.choice(C, size=L, replace=False) for L in lens]).astype(np.int32)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    p = ebic.Params.make(neg_trends=1, ratio_num=85, ratio_den=100, mode=ebic.MODE_AUTO)
    op = OParams(neg_trends=1, ratio_num=85, ratio_den=100, min_rows=p.min_rows, col_cap=p.col_cap)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x.copy())
        tune = ctx.autotune(ci, off, p, 100)
        before = ctx.profile_read(ebic.KERNEL_RANK_CODES)["launches"]
        built = ctx.profile_read(ebic.KERNEL_BITMAP_BUILD)["launches"]
        ctx.load_matrix(x)                                # (host, same shape: segmented)
        r_pad = (R + 127) // 128 * 128
        seg = max(8192, -(-((r_pad + 3) // 4) // 8192) * 8192)     # (four segments)
        assert ctx.profile_read(ebic.KERNEL_RANK_CODES)["launches"] - before == -(-r_pad // seg)
        assert ctx.profile_read(ebic.KERNEL_BITMAP_BUILD)["launches"] - built == \
            (1 if tune["mode"] == ebic.MODE_BITMAP else 0)
        got = ctx.eval_population(ci, off, p)
        if tune["mode"] == ebic.MODE_BITMAP:
            wst = r_pad // 32
            words = np.zeros(C * C * wst, np.uint32)
            ctx.copy_bitmap(words)
            cnt = np.zeros(C * C, np.uint64)
            ctx.copy_pair_counts(cnt)
            words = words.reshape(C, C, wst)
            cnt = cnt.reshape(C, C)
            W = (R + 31) // 32
            popc = lambda w: int(np.unpackbits(np.asarray(w, np.uint32).view(np.uint8)).sum())
            for a, b in [(0, 1), (C - 2, C - 1)] + [tuple(sorted(g.choice(C, 2, replace=False)))
                                                     for _ in range(40)]:
                wab, wba = pair_words(x, a, b), pair_words(x, b, a)
                assert np.array_equal(words[a, b, :W], wab) and np.array_equal(words[b, a, :W], wba)
                assert int(cnt[a, b]) == popc(wab) | (popc(wba) << 32)
    want = ocounts.eval_population(x, ci, off, op)
    for g_, w_ in zip(got, want):
        assert np.array_equal(np.asarray(g_, np.int64), np.asarray(w_, np.int64))

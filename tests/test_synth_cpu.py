"""The seeded input recipe (no GPU): workload shapes, planted structure, population ranges and
determinism, so that the tests and the benchmark measure the workloads the recipe defines."""

import numpy as np
import pytest

from paper_2105_01196_gb300 import synth

SHAPES = {  # name: (rows, cols, planted, population, lengths, ratio, negative trends)
    "tiny": (200, 20, 2, 64, (2, 6), (1, 1), 0),
    "default": (10_000, 100, 5, 800, (2, 20), (85, 100), 1),
    "batched": (20_000, 500, 10, 4096, (2, 64), (85, 100), 1),
    "tieheavy": (60_000, 1000, 20, 8192, (2, 64), (85, 100), 1),
}


@pytest.mark.parametrize("name", ["tiny", "default"])
def test_workload_shapes_and_population(name):
    rows, cols, n_bic, pop, (lo, hi), ratio, neg = SHAPES[name]
    w = synth.WORKLOADS[name]
    assert (w.rows, w.cols, w.n_bic, w.pop, w.len_lo, w.len_hi, w.ratio, w.neg_trends) == \
        (rows, cols, n_bic, pop, lo, hi, ratio, neg)
    x, truth, ci, off = synth.workload_inputs(w)
    assert x.shape == (rows, cols) and x.dtype == np.float32 and x.flags["C_CONTIGUOUS"]
    assert np.isfinite(x).all()
    assert len(truth) == n_bic
    lens = np.diff(off)
    assert len(lens) == pop and lens.min() >= lo and lens.max() <= hi
    assert off[0] == 0 and off[-1] == len(ci) and ci.dtype == np.int32
    for i in range(pop):
        c = ci[off[i]:off[i + 1]]
        assert len(set(c.tolist())) == len(c) and c.min() >= 0 and c.max() < cols


def test_larger_workload_parameters():
    for name in ("batched", "tieheavy"):
        rows, cols, n_bic, pop, (lo, hi), ratio, neg = SHAPES[name]
        w = synth.WORKLOADS[name]
        assert (w.rows, w.cols, w.n_bic, w.pop, w.len_lo, w.len_hi, w.ratio, w.neg_trends) == \
            (rows, cols, n_bic, pop, lo, hi, ratio, neg)
    t = synth.WORKLOADS["tieheavy"]
    assert (t.background, t.round_to) == ("lognormal", 0.1)


def test_planted_rows_follow_their_order():
    x, truth = synth.planted_matrix(500, 30, 4, (40, 60), (5, 8), seed=3, noise=0.0)
    seen_rows = set()
    for b, (ridx, order, sign) in reversed(list(enumerate(truth))):
        # later biclusters overwrite earlier ones: check rows no later bicluster touched, on the
        # columns no later bicluster took (with noise 0 every step increases by 0.5-1.5)
        target = order if sign > 0 else order[::-1]
        vals = x[np.ix_(ridx, target)]
        steps = np.diff(vals, axis=1)
        clean = [k for k, r in enumerate(ridx) if r not in seen_rows]
        if clean:
            assert (steps[clean] > 0.49).all() and (steps[clean] < 1.51).all()
        seen_rows.update(ridx.tolist())
    assert sum(1 for (_, _, s) in truth if s < 0) == 2   # neg_fraction 1/2


def test_log_normal_planted_rows_stay_ordered_and_positive():
    x, truth = synth.planted_matrix(400, 16, 3, (30, 40), (5, 8), seed=9, background="lognormal",
                                    noise=0.0)
    seen_rows = set()
    for ridx, order, sign in reversed(truth):
        target = order if sign > 0 else order[::-1]
        clean = [k for k, r in enumerate(ridx) if r not in seen_rows]
        vals = x[np.ix_(ridx[clean], target)]
        assert (vals > 0).all() and (np.diff(vals, axis=1) > 0.49).all()
        seen_rows.update(ridx.tolist())


def test_tie_heavy_background_is_rounded():
    x, _ = synth.planted_matrix(300, 12, 1, (20, 20), (4, 4), seed=5, background="lognormal",
                                round_to=0.1)
    assert np.allclose(x * 10, np.round(x * 10), atol=1e-4)
    # many ties within a row
    assert np.mean([len(np.unique(r)) < len(r) for r in x]) > 0.5


def test_inputs_are_deterministic_and_seed_dependent():
    w = synth.WORKLOADS["tiny"]
    a = synth.workload_inputs(w)
    b = synth.workload_inputs(w)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[2], b[2])
    c = synth.planted_matrix(200, 20, 2, (30, 30), (5, 5), seed=w.seed + 1, neg_fraction=0.0)
    assert not np.array_equal(a[0], c[0])

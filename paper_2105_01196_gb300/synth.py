"""Seeded synthetic inputs: planted trend-bicluster matrices and random populations.

This module holds none of the method's arithmetic: it only draws inputs.  The tests, the smoke
check and the benchmark use it for both the CUDA path and the CPU oracle, which then share the
same inputs and nothing else.

Recipe (stands in for the paper's Unibic / RecBic collections, Sec. 2.1, which are not shipped):
  * background N(0, 1) float32 (or log-normal(0, 1) rounded to 0.1 for the tie-heavy workload);
  * each planted bicluster takes rows and columns without replacement; its column order is a
    random permutation; a planted row gets s ~ N(0, 1) at the first column of the order and adds
    an increment ~ U(0.5, 1.5) at each next column, plus N(0, 0.1) noise per entry (on the
    log-normal background the row is then shifted to start at exp(s), keeping its order); a
    negative bicluster stores the values along the reversed order; later biclusters overwrite
    earlier ones;
  * a population has lengths uniform in [len_lo, len_hi] and distinct columns drawn uniformly.
Generators are numpy ``Generator(Philox(seed))``.
"""

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20210710


@dataclass
class Workload:
    name: str
    rows: int
    cols: int
    n_bic: int
    bic_rows: tuple
    bic_cols: tuple
    pop: int
    len_lo: int
    len_hi: int
    ratio: tuple          # (num, den)
    neg_trends: int
    generations: int
    background: str = "normal"
    round_to: float = 0.0
    neg_fraction: float = 0.5
    seed: int = SEED_BASE
    extra: dict = field(default_factory=dict)


# The five workload shapes of the evaluation: tiny, default scale, batched, tie-heavy, serving.
WORKLOADS = {
    "tiny": Workload("tiny", 200, 20, 2, (30, 30), (5, 5), 64, 2, 6, (1, 1), 0, 1,
                     neg_fraction=0.0, seed=SEED_BASE + 0),
    "default": Workload("default", 10_000, 100, 5, (100, 500), (5, 20), 800, 2, 20, (85, 100), 1,
                        100, seed=SEED_BASE + 1),
    "batched": Workload("batched", 20_000, 500, 10, (50, 2000), (5, 40), 4096, 2, 64, (85, 100),
                        1, 200, seed=SEED_BASE + 2),
    "tieheavy": Workload("tieheavy", 60_000, 1000, 20, (100, 5000), (5, 50), 8192, 2, 64,
                         (85, 100), 1, 100, background="lognormal", round_to=0.1,
                         seed=SEED_BASE + 3),
}


# The job stream of the serving workload: 256 jobs, Poisson arrivals at 20 jobs/s, matrices of
# 1,000-50,000 rows x 20-500 columns with 3-10 planted biclusters, population 800, ratio 0.85,
# 50 generations.
SERVING = dict(n_jobs=256, rate_per_s=20.0, rows=(1_000, 50_000), cols=(20, 500), n_bic=(3, 10),
               pop=800, ratio=(85, 100), generations=50, seed=SEED_BASE + 4)


def serving_stream(n_jobs=None, seed=None):
    """Arrival times (s), shapes and run seeds of the serving stream, and a generator of each
    job's matrix: a fresh shape per job (rows and columns uniform in the stream's ranges), its
    N(0, 1) background a crop at a random offset of one pre-drawn 50,000 x 500 pool (drawing 256
    fresh backgrounds of up to 25M values would take longer than the stream), with the job's own
    3-10 planted biclusters.  Returns (jobs, make) with jobs = [(arrival_s, rows, cols, seed)]
    and make(k) -> float32 [rows, cols] of job k."""
    cfg = SERVING
    n_jobs = cfg["n_jobs"] if n_jobs is None else n_jobs
    g = rng(cfg["seed"] if seed is None else seed)
    pool = g.standard_normal((cfg["rows"][1], cfg["cols"][1]), dtype=np.float32)
    gaps = g.exponential(1.0 / cfg["rate_per_s"], size=n_jobs)
    arrivals = np.cumsum(gaps) - gaps[0]
    jobs, spec = [], []
    for k in range(n_jobs):
        R = int(g.integers(cfg["rows"][0], cfg["rows"][1] + 1))
        C = int(g.integers(cfg["cols"][0], cfg["cols"][1] + 1))
        r_off = int(g.integers(0, cfg["rows"][1] - R + 1))
        c_off = int(g.integers(0, cfg["cols"][1] - C + 1))
        nb = int(g.integers(cfg["n_bic"][0], cfg["n_bic"][1] + 1))
        jobs.append((float(arrivals[k]), R, C, int(g.integers(1 << 31))))
        spec.append((r_off, c_off, nb, int(g.integers(1 << 31))))

    def make(k):
        _, R, C, _ = jobs[k]
        r_off, c_off, nb, pseed = spec[k]
        x = np.array(pool[r_off:r_off + R, c_off:c_off + C], dtype=np.float32, order="C")
        plant(x, nb, (max(10, R // 100), max(20, R // 20)), (4, min(20, C // 2)), rng(pseed))
        return x
    return jobs, make


def serving_jobs(n_jobs=None, n_matrices=16, seed=None):
    """Arrival times (s) and (matrix index, run seed) of the serving stream, and its matrices.

    Generating a new 50,000 x 500 matrix per job would take longer than the arrivals leave, so
    the stream draws its jobs' matrices from `n_matrices` pre-generated ones of random shape; each
    job has its own EBIC seed."""
    cfg = SERVING
    n_jobs = cfg["n_jobs"] if n_jobs is None else n_jobs
    g = rng(cfg["seed"] if seed is None else seed)
    mats = []
    for m in range(n_matrices):
        R = int(g.integers(cfg["rows"][0], cfg["rows"][1] + 1))
        C = int(g.integers(cfg["cols"][0], cfg["cols"][1] + 1))
        nb = int(g.integers(cfg["n_bic"][0], cfg["n_bic"][1] + 1))
        x, _ = planted_matrix(R, C, nb, (max(10, R // 100), max(20, R // 20)),
                              (4, min(20, C // 2)), seed=int(g.integers(1 << 31)))
        mats.append(x)
    gaps = g.exponential(1.0 / cfg["rate_per_s"], size=n_jobs)
    arrivals = np.cumsum(gaps) - gaps[0]
    jobs = [(float(arrivals[k]), int(g.integers(n_matrices)), int(g.integers(1 << 31)))
            for k in range(n_jobs)]
    return jobs, mats


def rng(seed):
    return np.random.Generator(np.random.Philox(int(seed)))


def planted_matrix(rows, cols, n_bic, bic_rows, bic_cols, seed, background="normal",
                   round_to=0.0, neg_fraction=0.5, noise=0.1):
    """Returns (x float32 [rows, cols] row-major, truth list of (row_idx, col_order, sign))."""
    g = rng(seed)
    if background == "normal":
        x = g.standard_normal((rows, cols), dtype=np.float32)
    elif background == "lognormal":
        x = g.lognormal(0.0, 1.0, size=(rows, cols)).astype(np.float32)
    else:
        raise ValueError(background)
    truth = plant(x, n_bic, bic_rows, bic_cols, g, background, neg_fraction, noise)
    if round_to:
        x = (np.round(x / round_to) * round_to).astype(np.float32)
    return np.ascontiguousarray(x, dtype=np.float32), truth


def plant(x, n_bic, bic_rows, bic_cols, g, background="normal", neg_fraction=0.5, noise=0.1):
    """Plants n_bic trend biclusters into x in place (recipe in the module docstring); returns
    their truth list of (row_idx, col_order, sign)."""
    rows, cols = x.shape
    truth = []
    n_neg = int(round(n_bic * neg_fraction))
    for b in range(n_bic):
        nr = int(g.integers(bic_rows[0], bic_rows[1] + 1))
        nc = int(g.integers(bic_cols[0], bic_cols[1] + 1))
        nr, nc = min(nr, rows), min(nc, cols)
        ridx = np.sort(g.choice(rows, size=nr, replace=False))
        order = g.choice(cols, size=nc, replace=False)
        sign = -1 if b < n_neg else 1
        start = g.standard_normal(nr)
        steps = g.uniform(0.5, 1.5, size=(nr, nc - 1))
        vals = np.concatenate([start[:, None], start[:, None] + np.cumsum(steps, axis=1)], axis=1)
        vals = vals + g.normal(0.0, noise, size=(nr, nc))
        if background == "lognormal":
            # onto the positive log-normal scale by a per-row shift, which keeps each row's order
            vals = vals - vals.min(axis=1, keepdims=True) + np.exp(start)[:, None]
        target = order if sign > 0 else order[::-1]
        x[np.ix_(ridx, target)] = vals.astype(np.float32)
        truth.append((ridx, np.asarray(order), sign))
    return truth


def random_population(n_ind, cols, len_lo, len_hi, seed):
    """CSR population: (col_idx int32 [sum L], offsets int32 [n_ind + 1])."""
    g = rng(seed)
    lens = g.integers(len_lo, len_hi + 1, size=n_ind)
    offsets = np.zeros(n_ind + 1, dtype=np.int32)
    offsets[1:] = np.cumsum(lens)
    col_idx = np.empty(int(offsets[-1]), dtype=np.int32)
    for i, L in enumerate(lens):
        col_idx[offsets[i]:offsets[i + 1]] = g.choice(cols, size=int(L), replace=False)
    return col_idx, offsets


def workload_inputs(w):
    """Matrix, ground truth and evaluation population of a named workload."""
    x, truth = planted_matrix(w.rows, w.cols, w.n_bic, w.bic_rows, w.bic_cols, w.seed,
                              background=w.background, round_to=w.round_to,
                              neg_fraction=w.neg_fraction)
    col_idx, offsets = random_population(w.pop, w.cols, w.len_lo, w.len_hi, w.seed + 1000)
    return x, truth, col_idx, offsets

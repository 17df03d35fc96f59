"""EBIC parameters (Sec. 2.4, last paragraph: negative trends on/off, approximate-trend threshold,
allowed overlap, number of iterations and of biclusters; Table 1: ``-n 20000``).

The paper names these parameters but gives no defaults other than the iteration cap.  The defaults
below are readings of the paper, one per parameter:
  ratio_num/ratio_den  approximate-trend ratio as a rational; 1/1 is the exact trend.
  min_rows             fewer accepted rows than this gives fitness 0.
  col_cap              fitness column exponent cap.
  overlap_num/den      allowed column overlap of a top-list entry with any better entry.
  init_min_len/max     initial chromosome length range (Sec. 2.4, step 1, "short chromosomes").
  elite                number of top-list entries copied into each new population (step 4).
  tournament           tournament size (step 5).
  max_attempts         children tried per slot before the slot is declared dead (tabu, step 5).
  tabu_hit_limit       per-generation tabu hits that stop the run (step 6); <= 0 disables.
  non_strict           1: ties count as following both directions (pair test >= / <=).
  last_kept            1: compare each value with the last value that kept the trend.

Test infrastructure only (see the package docstring).
"""

from dataclasses import dataclass, asdict

MAX_LEN = 64


@dataclass
class Params:
    neg_trends: int = 1
    ratio_num: int = 85
    ratio_den: int = 100
    min_rows: int = 2
    col_cap: int = 10
    overlap_num: int = 1
    overlap_den: int = 2
    n_biclusters: int = 10
    init_min_len: int = 2
    init_max_len: int = 8
    max_len: int = 20
    pop_size: int = 800
    elite: int = 10
    tournament: int = 4
    max_attempts: int = 4
    tabu_hit_limit: int = 800
    seed: int = 20210710
    non_strict: int = 0
    last_kept: int = 0

    def as_dict(self):
        return asdict(self)


def validate(p, n_cols):
    """Raise ValueError on a parameter set the method cannot run with."""
    if not (0 < p.ratio_num <= p.ratio_den):
        raise ValueError("ratio must satisfy 0 < ratio_num <= ratio_den")
    if not (p.overlap_den > 0 and 0 <= p.overlap_num <= p.overlap_den):
        raise ValueError("overlap must satisfy 0 <= overlap_num <= overlap_den, overlap_den > 0")
    if not (2 <= p.init_min_len <= p.init_max_len <= p.max_len <= min(MAX_LEN, n_cols)):
        raise ValueError("need 2 <= init_min_len <= init_max_len <= max_len <= min(64, cols)")
    if not (1 <= p.n_biclusters <= 256):
        raise ValueError("n_biclusters must be in [1, 256]")
    if not (2 <= p.pop_size <= (1 << 20)):
        raise ValueError("pop_size must be in [2, 2^20]")
    if not (0 <= p.elite <= p.n_biclusters and p.elite < p.pop_size):
        raise ValueError("elite must be in [0, min(n_biclusters, pop_size - 1)]")
    if not (1 <= p.tournament <= 16 and 1 <= p.max_attempts <= 16):
        raise ValueError("tournament and max_attempts must be in [1, 16]")
    if not (0 <= p.col_cap <= 16 and p.min_rows >= 0):
        raise ValueError("col_cap must be in [0, 16] and min_rows >= 0")
    if p.non_strict not in (0, 1) or p.last_kept not in (0, 1):
        raise ValueError("non_strict and last_kept are 0 or 1")

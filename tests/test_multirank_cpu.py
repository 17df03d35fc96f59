"""Multi-rank host logic on CPU (world size 2, gloo, 127.0.0.1), no GPU.

* bench.py's whole-job reduction: the slowest rank's time and the sum of all ranks' units (each
  rank runs an independent job; nothing else is exchanged).
* The row-sharded design for one large job (the paper's multi-GPU future work): trend counts are
  sums over rows, so per-shard counts summed by an all-reduce equal the whole matrix's counts,
  and the fitness computed from the summed counts equals the whole matrix's fitness.  Checked
  with the oracle on each rank's row shard."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            init_method=f"tcp://127.0.0.1:{port}")


def _reduce_worker(rank, world, port):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    _init(rank, world, port)
    try:
        ms, units = bench.reduce_over_ranks(dist, 10.0 + rank, 100.0 * (rank + 1), "cpu")
        assert (ms, units) == (11.0, 300.0), (ms, units)
    finally:
        dist.destroy_process_group()


def _shard_worker(rank, world, port):
    import sys
    sys.path.insert(0, ROOT)
    from oracle import counts
    from oracle.params import Params
    from paper_2105_01196_gb300 import synth
    _init(rank, world, port)
    try:
        x, _ = synth.planted_matrix(1001, 30, 3, (50, 200), (4, 10), seed=5)
        ci, off = synth.random_population(64, 30, 2, 20, seed=6)
        for ns, lk in ((0, 0), (1, 1)):
            p = Params(neg_trends=1, ratio_num=85, ratio_den=100, non_strict=ns, last_kept=lk)
            bounds = np.linspace(0, x.shape[0], world + 1).astype(int)   # uneven row shards
            shard = x[bounds[rank]:bounds[rank + 1]]
            mine = np.stack(counts.eval_population(shard, ci, off, p)[:3]).astype(np.int64)
            t = torch.from_numpy(mine)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            rp, rn, ra, f = counts.eval_population(x, ci, off, p)
            assert np.array_equal(t.numpy(), np.stack([rp, rn, ra]))
            lens = np.diff(off)
            f_from_sum = [counts.fitness(int(a), int(L), p.min_rows, p.col_cap)
                          for a, L in zip(t[2].tolist(), lens)]
            assert f_from_sum == [int(v) for v in f]
    finally:
        dist.destroy_process_group()


def test_bench_reduction_over_two_ranks():
    mp.spawn(_reduce_worker, args=(2, free_port()), nprocs=2, join=True)


def test_row_sharded_counts_sum_to_whole_matrix():
    mp.spawn(_shard_worker, args=(2, free_port()), nprocs=2, join=True)

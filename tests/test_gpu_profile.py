"""Kernel statistics (ebic_profile_*): event-timed launches of the evaluation and generation
kernels, in graph replays and eagerly, with the evaluation's algorithmic bytes."""

import pytest

from paper_2105_01196_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("use_graph,fuse", [(1, 63), (0, 63), (1, -1), (1, 0)])
def test_generation_kernels_are_timed(use_graph, fuse):
    """The evaluations the evolve kernel does itself (fuse_pairs) count as its work; the
    evaluation launches count the rest.  (0, the library's choice: none for 64 slots, one block
    per slot.)"""
    from paper_2105_01196_gb300 import ebic
    x, _, _, _ = synth.workload_inputs(synth.WORKLOADS["tiny"])
    p = ebic.Params.make(max_len=6, init_max_len=6, pop_size=64, elite=4, n_biclusters=4,
                         tabu_hit_limit=0, mode=ebic.MODE_BITMAP, use_graph=use_graph,
                         fuse_pairs=fuse)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        ctx.run_generations(p, 2)
        ctx.profile_enable(True)
        rep0 = ctx.run_generations(p, 0)
        ctx.run_generations(p, 6)
        rep = ctx.run_generations(p, 0)
        ev = ctx.profile_read(ebic.KERNEL_EVAL)
        evo = ctx.profile_read(ebic.KERNEL_EVOLVE)
        fin = ctx.profile_read(ebic.KERNEL_FINISH)
        ctx.profile_enable(False)
    assert ev["timed_launches"] == evo["timed_launches"] == fin["timed_launches"] == 6
    assert ev["ms"] > 0 and evo["ms"] > 0 and fin["ms"] > 0
    wst = ((x.shape[0] + 127) // 128) * 4
    fused = rep.n_fused - rep0.n_fused
    assert (fused > 0) == (fuse > 0)
    assert ev["units"] == (rep.n_evaluated - rep0.n_evaluated - fused) * x.shape[0]
    assert evo["units"] == fused * x.shape[0]
    assert ev["alg_bytes"] > 0 and ev["alg_bytes"] % (wst * 4) == 0
    # (one-pair slots scored from the pair-count table read one count per direction)
    ntab = rep.n_table - rep0.n_table
    words = evo["alg_bytes"] - ntab * 4 * (2 if p.neg_trends else 1)
    assert words % (wst * 4) == 0 and (evo["alg_bytes"] > 0) == (fuse > 0)
    assert (ntab > 0) == (fuse > 0)

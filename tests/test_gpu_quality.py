"""Search quality through the C ABI: the device generation loop on an easy planted matrix gives
the oracle's top list, hence the same clustering error (CE, Eq. 1) against the planted truth."""

import numpy as np
import pytest

from oracle import ebic as oebic
from oracle.params import Params as OParams
from oracle.quality import clustering_error as ce_oracle
from paper_2105_01196_gb300 import synth
from paper_2105_01196_gb300.quality import clustering_error as ce_package, rows_from_mask

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [1, 2])
def test_planted_recovery_ce_matches_oracle(mode):
    from paper_2105_01196_gb300 import ebic
    x, truth = synth.planted_matrix(160, 10, 1, (40, 40), (4, 4), seed=77, neg_fraction=0.0)
    base = dict(neg_trends=0, ratio_num=1, ratio_den=1, max_len=5, init_min_len=2,
                init_max_len=4, pop_size=48, elite=4, n_biclusters=4, tabu_hit_limit=0, seed=4)
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        ctx.run_generations(ebic.Params.make(mode=mode, **base), 40)
        top = ctx.toplist()
        masks = ctx.extract_biclusters(x.shape[0])
    op = OParams(**base)
    st = oebic.run(x, op, 40)
    want = oebic.extract(x, st, op)
    assert np.array_equal(masks[:, :want.shape[1]], want)
    found = [(rows_from_mask(masks[k], x.shape[0]), list(e["cols"])) for k, e in enumerate(top)]
    ref = [(r, o) for r, o, _ in truth]
    d, u, _, score = ce_oracle(found, ref)
    got = ce_package(found, ref, *x.shape)
    assert (got["d_max"], got["union"]) == (d, u)
    best = ce_package(found[:1], ref, *x.shape)
    assert best["score"] >= 0.8

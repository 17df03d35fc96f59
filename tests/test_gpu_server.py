"""Continuous-batching job server: jobs admitted by device-memory footprint and overlapping on the
GPU give the same results as the same jobs run alone (tolerance 0), including the oracle's."""

import time

import numpy as np
import pytest

from oracle import ebic as oebic
from oracle.params import Params as OParams
from paper_2105_01196_gb300 import synth

pytestmark = pytest.mark.gpu

BASE = dict(neg_trends=1, ratio_num=85, ratio_den=100, max_len=8, init_min_len=2, init_max_len=8,
            pop_size=128, elite=5, n_biclusters=5, tabu_hit_limit=0)


def make_jobs():
    jobs = []
    shapes = [(300, 20), (2000, 40), (1000, 30), (5000, 60), (400, 25), (3000, 50)]
    for k, (R, C) in enumerate(shapes):
        x, _ = synth.planted_matrix(R, C, 3, (20, min(200, R // 4)), (4, 8), seed=500 + k)
        jobs.append((x, dict(BASE, seed=1000 + k), 6 + 2 * k))
    return jobs


def alone(ebic, x, kw, n_gen):
    with ebic.Context(0) as ctx:
        ctx.load_matrix(x)
        rep = ctx.run_generations(ebic.Params.make(**kw), n_gen)
        return rep, ctx.toplist()


def test_jobs_in_the_mix_equal_jobs_alone():
    from paper_2105_01196_gb300 import ebic
    jobs = make_jobs()
    refs = [alone(ebic, x, kw, n) for x, kw, n in jobs]
    fps = sorted(ebic.ebic_job_footprint(x.shape[0], x.shape[1], ebic.Params.make(**kw), n)
                 for x, kw, n in jobs)
    budget = fps[-1] + fps[-2]        # every job fits; several of the smaller ones run together
    with ebic.Server(0, hbm_budget_bytes=budget, max_running=3) as srv:
        ids = [srv.submit(x, ebic.Params.make(**kw), n) for x, kw, n in jobs]
        peak = 0
        for _ in range(200):
            st = srv.stats()
            peak = max(peak, st["running"])
            assert st["reserved"] <= budget and st["running"] <= 3
            if st["running"] == 0 and st["queued"] == 0:
                break
            time.sleep(0.002)
        results = [srv.wait(j) for j in ids]
    for (rep, top), res in zip(refs, results):
        assert res["status"] == ebic.EBIC_OK
        assert res["gens_done"] == rep.gens_done and res["n_evaluated"] == rep.n_evaluated
        assert res["top"] == top


def test_small_job_matches_oracle():
    from paper_2105_01196_gb300 import ebic
    x, _, _, _ = synth.workload_inputs(synth.WORKLOADS["tiny"])
    kw = dict(BASE, max_len=6, init_max_len=6, pop_size=64, elite=4, n_biclusters=4, seed=21)
    with ebic.Server(0, hbm_budget_bytes=1 << 30, max_running=2) as srv:
        res = srv.wait(srv.submit(x, ebic.Params.make(**kw), 15))
    st = oebic.run(x, OParams(**kw), 15)
    assert res["gens_done"] == st.gen
    assert [(e["cols"], e["f"], e["h"]) for e in res["top"]] == \
        [(tuple(e.cols), e.f, e.h) for e in st.top]


def test_admission_limits():
    from paper_2105_01196_gb300 import ebic
    x, _ = synth.planted_matrix(4000, 60, 2, (50, 100), (4, 6), seed=7)
    p = ebic.Params.make(**dict(BASE, seed=3))
    fp = ebic.ebic_job_footprint(4000, 60, p, 30)
    assert fp > 4000 * 60 * 4
    with ebic.Server(0, hbm_budget_bytes=fp + fp // 2, max_running=4) as srv:
        with pytest.raises(ebic.EbicError) as e:
            srv.submit(np.zeros((20000, 200), np.float32), p, 30)   # never fits the budget
        assert e.value.code == ebic.EBIC_ENOMEM
        ids = [srv.submit(x, p, 30) for _ in range(3)]
        seen_running = 0
        for _ in range(500):
            st = srv.stats()
            seen_running = max(seen_running, st["running"])
            assert st["running"] <= 1                     # only one job fits at a time
            if st["running"] == 0 and st["queued"] == 0:
                break
            time.sleep(0.001)
        res = [srv.wait(j) for j in ids]
        assert all(r["status"] == ebic.EBIC_OK for r in res)
        assert res[0]["top"] == res[1]["top"] == res[2]["top"]     # same job, same result

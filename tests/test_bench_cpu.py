"""bench.py's host-side measurement helpers, on CPU: the committed ncu traffic summary it reads,
the kernel a form runs, the peak it divides by, the single-thread oracle baseline, and the shape
of the reference arm's JSON line."""

import json
import os

import numpy as np
import pytest

import bench
from paper_2105_01196_gb300 import synth


def test_ncu_traffic_reads_the_committed_summary():
    """Each committed row is read with its source; a row whose kernel source has changed since
    its capture is reported stale (no traffic), a current one within the expected bounds."""
    def fresh_or_stale(kernel, workload, lo, hi):
        v, src = bench.ncu_traffic_entry(kernel, workload)
        assert src is not None and f"traffic_{kernel}.txt" in src and "commit" in src
        if v is None:
            assert "stale" in src
        else:
            assert lo < v < hi
    # DRAM bytes per launch stay below the algorithmic bytes (part of the pair words hit L2;
    # the loop launches' mean includes the initial population's full sweep)
    fresh_or_stale("k_eval_bitmap", "default-loop", 0, 5.39e6)  # (the bitmap stays in L2)
    fresh_or_stale("k_eval_bitmap", "tieheavy-loop", 3e7, 1.3e8)
    fresh_or_stale("k_evolve_seq", "tieheavy-loop", 3e7, 1.3e8)
    assert bench.ncu_traffic("k_eval_bitmap", "no-such-workload") is None
    assert bench.ncu_traffic("no_such_kernel", "default") is None


def test_ncu_traffic_row_goes_stale_with_its_kernel_source(tmp_path, monkeypatch):
    """A summary row counts only while the hash of its kernel's source files matches: the same
    files give the traffic, an edited file (or a row without a hash) gives none."""
    csrc = tmp_path / "paper_2105_01196_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    for f in bench.KERNEL_SOURCES["k_evolve_seq"]:
        with open(os.path.join(bench.ROOT, "paper_2105_01196_gb300", "csrc", f), "rb") as fh:
            (csrc / f).write_bytes(fh.read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_source_hash("k_evolve_seq")
    assert h is not None and len(h) == 12
    row = tmp_path / "profiles" / "traffic_k_evolve_seq.txt"
    row.write_text(f"# header\nk_evolve_seq w1 1000 abc1234 {h}\nk_evolve_seq w2 2000 abc1234\n")
    assert bench.ncu_traffic_entry("k_evolve_seq", "w1")[0] == 1000.0
    v, src = bench.ncu_traffic_entry("k_evolve_seq", "w2")
    assert v is None and "stale" in src
    with open(csrc / "evolve.cu", "ab") as fh:
        fh.write(b"\n// edited\n")
    assert bench.kernel_source_hash("k_evolve_seq") != h
    v, src = bench.ncu_traffic_entry("k_evolve_seq", "w1")
    assert v is None and "stale" in src and "abc1234" in src


def test_eval_kernel_names():
    assert bench.eval_kernel_name(2, 100) == "k_eval_bitmap"
    assert bench.eval_kernel_name(1, 1024) == "k_eval_codes"
    assert bench.eval_kernel_name(1, 1025) == "k_eval_direct"
    assert bench.eval_kernel_name(4, 100) == "k_eval_direct_tma"
    assert bench.eval_kernel_name(3, 100) == "k_eval_plain"


def test_peak_is_the_measured_copy_bandwidth():
    peak, kind = bench.load_peaks()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            assert (peak, kind) == (json.load(fh)["hbm_gbs"], "measured")
    else:
        assert kind == "fallback"
    assert peak > 0


def test_cpu_baseline_counts_oracle_evaluations():
    w = synth.WORKLOADS["tiny"]
    x, _, ci, off = synth.workload_inputs(w)
    r = bench.cpu_baseline(w, x, ci, off, 0.2)
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["unit"] == bench.UNIT
    done = int(r["sample"].split("oracle trend counts of ")[1].split()[0])
    assert done >= 1 and r["value"] > 0
    assert f"x {x.shape[0]} rows" in r["sample"]


def test_cpu_baseline_pool_uses_every_core_and_matches_the_serial_oracle():
    """The pool's counts map gives the serial oracle's run exactly (it only moves the
    independent per-individual counts to other processes), and the baseline reports the cores
    from the affinity mask and the oracle's generations per second."""
    import dataclasses
    from oracle import ebic as oebic
    from oracle.params import Params as OParams
    w = dataclasses.replace(synth.WORKLOADS["tiny"], generations=3)
    x, _, ci, off = synth.workload_inputs(w)
    fields = bench.run_fields(w)
    with bench.OraclePool(x) as pool:
        assert pool.cores == len(os.sched_getaffinity(0))
        r = bench.cpu_baseline(w, x, ci, off, 0.3, pool=pool, generation=True)
        a = oebic.run(x, OParams(**fields), 3, counts_map=pool.counts_map(fields))
    b = oebic.run(x, OParams(**fields), 3)
    assert [(e.cols, e.f, e.h) for e in a.top] == [(e.cols, e.f, e.h) for e in b.top]
    assert a.pop == b.pop and a.fit == b.fit and a.rows == b.rows and a.hits == b.hits
    assert r["cores"] == pool.cores and r["value"] > 0 and r["generations_per_s"] > 0
    assert "1 generation timed" in r["generation_sample"]


def test_reference_arm_line(monkeypatch, capsys):
    calls = []

    def fake_baseline(w, x, ci, off, seconds, trend="strict", pool=None):
        calls.append(seconds)
        return {"value": float(len(calls)), "unit": bench.UNIT, "cores": 1, "kind": "oracle",
                "sample": "stub"}

    monkeypatch.setattr(bench, "cpu_baseline", fake_baseline)

    class Args:
        steps, warmup, gpus, gens, mode, trend, pool = 3, 3, 1, None, "auto", "strict", False

    bench.run_reference(Args, synth.WORKLOADS["tiny"], 1, 0, None)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True
    # the median of the timed steps (values 4, 5, 6 after three warm-up calls)
    assert line["value"] == pytest.approx(5.0)
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == 5.0
    assert line["e2e"] == {"value": 5.0, "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert len(calls) == 6 and calls[0] == pytest.approx(calls[-1] / 4)
    # a rank other than 0 prints nothing
    bench.run_reference(Args, synth.WORKLOADS["tiny"], 2, 1, None)
    assert capsys.readouterr().out == ""
    assert np.isfinite(line["ms_per_step"])

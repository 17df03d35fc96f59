"""EBIC population-evaluation benchmark on GB300.

One step = one pass of the whole hot path over one synthetic workload, through the C ABI:
  matrix upload (order keys) -> pair-bitmap build (when the autotuner picks the bitmap form)
  -> full evaluation of the workload's population -> the EBIC generation loop (initial
  population + `--gens` generations, graph-replayed) -> bicluster extraction of the top list.
The metric is (individual, row) trend evaluations per second over the step; generations per
second are reported beside it.  Default workload: 10,000 x 100 float32, population 800, lengths
2-20, approximate ratio 0.85, negative trends, 100 generations.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload default|tiny|batched|tieheavy] [--gens G] [--mode auto|...]
Multi-GPU (torchrun): every rank runs an independent job (its own seed) on its own GPU; the
value is all ranks' evaluations divided by the slowest rank's time ("weak" scaling).
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "individual·row trend evaluations/sec and EBIC generations/sec vs plain GPU form"
UNIT = "evals/s"
MODES = {"auto": 0, "direct": 1, "bitmap": 2, "plain": 3, "staged": 4}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="default")
    ap.add_argument("--gens", type=int, default=None, help="generations per step")
    ap.add_argument("--mode", default="auto", choices=list(MODES))
    ap.add_argument("--trend", default="strict",
                    choices=["strict", "ties", "last-kept", "ties-last-kept"],
                    help="pair test: strict (default), ties holding for both directions, "
                         "comparison with the last kept value, or both")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-scale-roofline", action="store_true",
                    help="skip the evaluation-kernel roofline on the batched workload")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--jobs", type=int, default=0, help="serving: number of jobs (0 = 256)")
    ap.add_argument("--max-running", type=int, default=8, help="serving: concurrent jobs")
    return ap.parse_args()


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local, dist


def gens_of(args, w):
    return w.generations if args.gens is None else args.gens


def reduce_over_ranks(dist, total_ms, units, device):
    """Whole-job timing over the ranks: the slowest rank's time and the sum of all ranks' units
    (each rank runs an independent job, so nothing else is exchanged)."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.barrier()
    return float(t.item()), float(u.item())


def search_quality(ctx, truth, R, C, gens):
    """CE (Eq. 1) of the last run's top list, with the rows that follow each entry, against the
    planted biclusters (measured after the timed region)."""
    from paper_2105_01196_gb300.quality import clustering_error, rows_from_mask
    top = ctx.toplist()
    masks = ctx.extract_biclusters(R)
    found = [(rows_from_mask(masks[k], R), list(e["cols"])) for k, e in enumerate(top)]
    ref = [(rows, order) for rows, order, _ in truth]
    ce = clustering_error(found, ref, R, C)
    # for each planted bicluster, the best pairwise CE score over the found entries
    best = [max((clustering_error([f], [t], R, C)["score"] for f in found), default=0.0)
            for t in ref]
    return {"ce_score": ce["score"], "ce_error": ce["error"], "d_max": ce["d_max"],
            "union": ce["union"], "found": len(found), "planted": len(ref),
            "best_pair_score_per_planted": [round(b, 4) for b in best],
            "generations": gens, "measure": "clustering error, Eq. 1 (Munkres assignment); "
            "score = D_max/|U|, 1 = perfect"}


def eval_kernel_name(mode, cols):
    """The evaluation kernel a form runs (the direct form reads rank codes up to 1,024 columns)."""
    if mode == 2:
        return "k_eval_bitmap"
    if mode == 4:
        return "k_eval_direct_tma"
    if mode == 3:
        return "k_eval_plain"
    if mode == 1:
        return "k_eval_codes" if cols <= 1024 else "k_eval_direct"
    return "k_eval_bitmap|k_eval_codes"


def scale_roofline(ebic, dev, stream, peak, peak_kind, sweeps=20):
    """The evaluation kernel on the batched workload (20,000 x 500, P 4,096, lengths 2-64, ratio
    0.85, negative trends), where a sweep is large enough to reach its memory bound: bitmap
    sweeps timed with CUDA events on the library stream after a warm-up sweep, outside the timed
    region of the step.  Algorithmic bytes as in the main roofline."""
    import torch
    from paper_2105_01196_gb300 import synth
    w = synth.WORKLOADS["batched"]
    x, _, ci, off = synth.workload_inputs(w)
    P = len(off) - 1
    xd = torch.from_numpy(x).to(dev)
    cid, offd = torch.from_numpy(ci).to(dev), torch.from_numpy(off).to(dev)
    outs = [torch.zeros(P, dtype=torch.int32, device=dev) for _ in range(3)]
    outs.append(torch.zeros(P, dtype=torch.int64, device=dev))
    p = ebic.Params.make(neg_trends=1, ratio_num=w.ratio[0], ratio_den=w.ratio[1], mode=2)
    with ebic.Context(dev.index or 0, stream.cuda_stream) as c:
        c.load_matrix(xd)
        c.build_bitmap()
        c.eval_population(cid, offd, p, *outs)
        c.profile_enable(True)
        for _ in range(sweeps):
            c.eval_population(cid, offd, p, *outs)
        st = c.profile_read(ebic.KERNEL_EVAL)
        c.profile_enable(False)
    avg_s = st["ms"] / st["timed_launches"] / 1e3
    per_launch = st["alg_bytes"] / st["timed_launches"]
    achieved = per_launch / avg_s / 1e9
    return {"workload": "batched", "kernel": "k_eval_bitmap", "bound": "hbm",
            "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": ncu_traffic("k_eval_bitmap", "batched"),
            "peak_kind": peak_kind, "alg_bytes_per_launch": per_launch,
            "avg_launch_us": avg_s * 1e6, "launches": st["timed_launches"],
            "note": "bitmap (628 MB) larger than L2, so no flush between sweeps; algorithmic "
                    "bytes count every pair word read, some of which individuals share"}


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu summary, or None."""
    path = os.path.join(ROOT, "profiles", "traffic_" + kernel + ".txt")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) == 3 and not line.startswith("#") and parts[:2] == [kernel, workload]:
                return float(parts[2])
    return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs"), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples taken while the timed region runs."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 3.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.01)          # first sample in before the timed region starts
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.05)                  # one more sample at the end of the timed region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def run_fields(w, trend="strict"):
    """The run parameters of a workload, shared by the GPU path and the oracle baseline."""
    return dict(neg_trends=w.neg_trends, ratio_num=w.ratio[0], ratio_den=w.ratio[1],
                pop_size=w.pop, max_len=min(w.len_hi, 64), init_min_len=w.len_lo,
                init_max_len=min(w.len_hi, 64), n_biclusters=max(10, w.n_bic),
                elite=max(10, w.n_bic), tabu_hit_limit=0, seed=w.seed,
                non_strict=int("ties" in trend), last_kept=int("last-kept" in trend))


# --------------------------------------------------------------------------- CPU oracle baseline
# The oracle runs unchanged; a process pool (started with "spawn", so no worker inherits a CUDA
# context) splits its independent per-individual trend counts over the host cores.  Workers map
# the matrix from a temporary .npy file instead of receiving a pickled copy.

_POOL_X = None


def _pool_init(path):
    global _POOL_X
    _POOL_X = np.load(path, mmap_mode="r")


def _pool_eval_timed(task):
    """Oracle trend counts of individuals start, start + stride, ... (cycling through the
    population) until `seconds` pass; returns how many were evaluated."""
    from oracle import counts as ocounts
    from oracle.params import Params as OParams
    ci, off, start, stride, seconds, fields = task
    p = OParams(**fields)
    n = len(off) - 1
    t0 = time.perf_counter()
    done, i = 0, start % n
    while time.perf_counter() - t0 < seconds:
        ocounts.eval_individual(_POOL_X, [int(c) for c in ci[off[i]:off[i + 1]]], p)
        done += 1
        i = (i + stride) % n
    return done


def _pool_counts(task):
    from oracle.ebic import row_counts
    from oracle.params import Params as OParams
    chroms, fields = task
    p = OParams(**fields)
    return [row_counts(_POOL_X, list(c), p) for c in chroms]


class OraclePool:
    """Worker processes on every core this process may run on (os.sched_getaffinity)."""

    def __init__(self, x):
        import multiprocessing as mp
        self.cores = len(os.sched_getaffinity(0))
        fd, self.path = tempfile.mkstemp(suffix=".npy")
        os.close(fd)
        np.save(self.path, np.ascontiguousarray(x))
        self.pool = mp.get_context("spawn").Pool(self.cores, initializer=_pool_init,
                                                 initargs=(self.path,))

    def counts_map(self, fields):
        """A counts_map for the oracle's scoring step: chromosomes split into one chunk per
        core, counted in the workers, returned in order."""
        def run(chroms):
            k = max(1, -(-len(chroms) // self.cores))
            chunks = [(chroms[i:i + k], fields) for i in range(0, len(chroms), k)]
            return [t for part in self.pool.map(_pool_counts, chunks) for t in part]
        return run

    def close(self):
        self.pool.terminate()
        self.pool.join()
        os.unlink(self.path)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def cpu_baseline(w, x, ci, off, seconds, trend="strict", pool=None, generation=False):
    """The CPU oracle as it stands, on a bounded sample of the workload: full trend counts of the
    workload's individuals, cycling through the population, for `seconds` (on every worker of
    `pool` at once, else single-threaded).  With `generation`, also one generation of the oracle's
    EBIC loop (initial population, then one timed generation, with the pool's counts map): the
    oracle's generations/s, measured on one generation of the workload's run."""
    from oracle import counts as ocounts
    from oracle.params import Params as OParams
    fields = run_fields(w, trend)
    n = len(off) - 1
    t0 = time.perf_counter()
    if pool is None:
        p = OParams(**fields)
        done = 0
        while time.perf_counter() - t0 < seconds:
            i = done % n
            ocounts.eval_individual(x, [int(c) for c in ci[off[i]:off[i + 1]]], p)
            done += 1
        cores = 1
    else:
        cores = pool.cores
        tasks = [(ci, off, k * (n // cores), 1, seconds, fields) for k in range(cores)]
        done = sum(pool.pool.map(_pool_eval_timed, tasks))
    dt = time.perf_counter() - t0
    out = {"value": done * x.shape[0] / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"oracle trend counts of {done} individual evaluations (the workload's "
                     f"{n} individuals, cycled) x {x.shape[0]} rows ({dt:.1f} s, "
                     + ("single thread)" if pool is None else
                        f"{cores} worker processes, individuals split over them)")}
    if generation:
        from oracle import ebic as oebic
        op = OParams(**fields)
        cmap = pool.counts_map(fields) if pool is not None else None
        t1 = time.perf_counter()
        st = oebic.initialise(x, op, cmap)
        t2 = time.perf_counter()
        oebic.next_generation(x, st, op, cmap)
        t3 = time.perf_counter()
        out["generations_per_s"] = 1.0 / (t3 - t2)
        out["generation_sample"] = (f"oracle EBIC loop on this workload: initial population "
                                    f"({t2 - t1:.1f} s) then 1 generation timed ({t3 - t2:.2f} s)"
                                    f" of the run's {w.generations}; "
                                    + ("single thread" if pool is None else
                                       f"trend counts on {cores} worker processes"))
    return out


def run_reference(args, w, world, rank, dist):
    """Reference arm: the CPU oracle on the host cores, each step a bounded sample."""
    from paper_2105_01196_gb300 import synth
    if rank != 0:
        return
    x, _, ci, off = synth.workload_inputs(w)
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    pool = OraclePool(x) if getattr(args, "pool", True) else None
    try:
        for _ in range(args.warmup):
            cpu_baseline(w, x, ci, off, per_step / 4, args.trend, pool=pool)
        vals = []
        t0 = time.perf_counter()
        last = None
        for _ in range(args.steps):
            last = cpu_baseline(w, x, ci, off, per_step, args.trend, pool=pool)
            vals.append(last["value"])
        total = time.perf_counter() - t0
    finally:
        if pool is not None:
            pool.close()
    v = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32-compare/int32",
            "data": "synthetic", "config": {"workload": w.name, "rows": w.rows, "cols": w.cols,
                                             "pop": w.pop, "len": [w.len_lo, w.len_hi],
                                             "ratio": list(w.ratio), "neg_trends": w.neg_trends,
                                             "generations": gens_of(args, w), "mode": args.mode,
                                             "trend": args.trend},
            "cpu_baseline": dict(last, value=v),
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args, world, rank, local, dist):
    """Serving workload: a Poisson stream of EBIC jobs through the continuous-batching server;
    p50/p99 job latency (arrival to completion) and jobs/s, plus the saturated throughput with
    every job queued at once."""
    import threading
    import torch
    from paper_2105_01196_gb300 import ebic, synth
    torch.cuda.set_device(local)
    cfg = synth.SERVING
    n_jobs = args.jobs if args.jobs else cfg["n_jobs"]
    jobs, mats = synth.serving_jobs(n_jobs, seed=cfg["seed"] + 7919 * rank)

    def params(seed):
        return ebic.Params.make(neg_trends=1, ratio_num=cfg["ratio"][0], ratio_den=cfg["ratio"][1],
                                pop_size=cfg["pop"], max_len=20, init_min_len=2, init_max_len=20,
                                n_biclusters=10, elite=10, tabu_hit_limit=0, seed=seed)
    free, total = torch.cuda.mem_get_info(local)
    budget = int(0.6 * free)
    out = {}
    for phase in ("poisson", "saturated"):
        lat = []
        evals = 0
        with ebic.Server(local, hbm_budget_bytes=budget, max_running=args.max_running) as srv:
            t0 = time.perf_counter()
            ids = []
            for at, m, seed in jobs:
                if phase == "poisson":
                    delay = t0 + at - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                ids.append((time.perf_counter(), srv.submit(mats[m], params(seed), cfg["generations"]), m))
            for t_sub, jid, m in ids:
                r = srv.wait(jid)
                assert r["status"] == 0, r
                lat.append(r["queued_ms"] + r["run_ms"])
                evals += r["n_evaluated"] * mats[m].shape[0]
            wall = time.perf_counter() - t0
        out[phase] = {"jobs_per_s": len(jobs) / wall, "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)), "wall_s": wall,
                      "evals_per_s": evals / wall}
    if rank == 0:
        line = {"metric": "EBIC jobs/sec and p50/p99 job latency (continuous batching)",
                "value": out["saturated"]["jobs_per_s"], "unit": "jobs/s", "n_gpus": world,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32-compare/int32", "data": "synthetic",
                "config": {"workload": "serving", "jobs": len(jobs), "rate_per_s": cfg["rate_per_s"],
                           "rows": list(cfg["rows"]), "cols": list(cfg["cols"]), "pop": cfg["pop"],
                           "generations": cfg["generations"], "distinct_matrices": len(mats),
                           "max_running": args.max_running, "hbm_budget_bytes": budget},
                "poisson": out["poisson"], "saturated": out["saturated"]}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local, dist = dist_setup(args)
    from paper_2105_01196_gb300 import synth
    import dataclasses
    if args.workload == "serving":
        run_serving(args, world, rank, local, dist)
        if dist:
            dist.destroy_process_group()
        return
    w = dataclasses.replace(synth.WORKLOADS[args.workload])
    if args.impl == "reference":
        run_reference(args, w, world, rank, dist)
        if dist:
            dist.destroy_process_group()
        return

    import torch
    from paper_2105_01196_gb300 import ebic
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    w = dataclasses.replace(w, seed=w.seed + 7919 * rank)
    gens = gens_of(args, w)
    x, truth, ci, off = synth.workload_inputs(w)
    R = w.rows
    x_d = torch.from_numpy(x).to(dev)
    ci_d = torch.from_numpy(ci).to(dev)
    off_d = torch.from_numpy(off).to(dev)
    P = len(off) - 1
    outs_d = [torch.zeros(P, dtype=torch.int32, device=dev) for _ in range(3)]
    outs_d.append(torch.zeros(P, dtype=torch.int64, device=dev))
    x_h = torch.from_numpy(x).pin_memory()
    outs_h = [torch.zeros(P, dtype=torch.int32).pin_memory() for _ in range(3)]
    outs_h.append(torch.zeros(P, dtype=torch.int64).pin_memory())
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    params = ebic.Params.make(mode=MODES[args.mode], **run_fields(w, args.trend))
    ctx = ebic.Context(local, stream.cuda_stream)
    used_mode = [0]                     # evaluation form the generation loop used

    def step(host):
        """One pass of the hot path; returns (individual,row) evaluations done."""
        units = 0
        if host:
            ctx.load_matrix(x_h)
            ctx.eval_population(ci, off, params, *outs_h)
        else:
            ctx.load_matrix(x_d)
            ctx.eval_population(ci_d, off_d, params, *outs_d)
        units += P * R
        if gens > 0:
            rep = ctx.run_generations(params, gens)
            used_mode[0] = int(rep.eval_mode)
            units += int(rep.n_evaluated) * R
            masks = ctx.extract_biclusters(R)
            units += len(masks) * R
        return units

    for _ in range(max(3, args.warmup)):
        step(False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ctx.profile_enable(True)            # reset the launch counters ...
    ctx.profile_enable(False)           # ... and time this pass without per-kernel events
    total_ms = 0.0
    units = 0
    for _ in range(args.steps):
        flush.zero_()                   # L2 flush between timed steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        units += step(False)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    st_all = ctx.profile_read(ebic.KERNEL_ALL)
    clk = clocks.stop()
    # Second pass over the same K steps with CUDA events around every kernel of the path
    # (event-record nodes inside the generation graphs): per-kernel durations and work.
    ctx.profile_enable(True)
    for _ in range(args.steps):
        flush.zero_()
        step(False)
    torch.cuda.synchronize()
    stats = {name: ctx.profile_read(kid) for name, kid in
             (("eval", ebic.KERNEL_EVAL), ("evolve", ebic.KERNEL_EVOLVE),
              ("finish", ebic.KERNEL_FINISH), ("bitmap_build", ebic.KERNEL_BITMAP_BUILD),
              ("rank_codes", ebic.KERNEL_RANK_CODES))}
    ctx.profile_enable(False)
    if dist:
        total_ms, units = reduce_over_ranks(dist, total_ms, units, dev)

    e2e = None
    if not args.no_e2e:
        # End to end through the same C ABI with host buffers: the copies run inside the calls.
        # Each step is timed on the host clock from a flushed L2, like the device-timed steps.
        e2e_units = 0
        e2e_s = 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_units += step(True)
            torch.cuda.synchronize()
            e2e_s += time.perf_counter() - t0
        h2d = x.nbytes + ci.nbytes + off.nbytes
        d2h = sum(o.numel() * o.element_size() for o in outs_h)
        if gens > 0:
            d2h += 256 * ((R + 127) // 128) * 16
        e2e = {"value": e2e_units / e2e_s * (world if dist else 1), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peak, peak_kind = load_peaks()
    timed_ms = sum(v["ms"] for v in stats.values())
    for v in stats.values():
        v["avg_us"] = 1e3 * v["ms"] / v["timed_launches"] if v["timed_launches"] else None
        v["share_of_kernel_time"] = v["ms"] / timed_ms if timed_ms else None
    dominant = max(stats, key=lambda k: stats[k]["ms"])
    kernel_names = {"eval": eval_kernel_name(used_mode[0] if used_mode[0] else MODES[args.mode],
                                             w.cols),
                    "evolve": "k_evolve", "finish": "k_finish", "bitmap_build": "k_build_bitmap",
                    "rank_codes": "k_rank_codes"}
    roof = None
    se = stats["eval"]
    if se["timed_launches"] > 0 and se["ms"] > 0:
        n_l = se["timed_launches"]
        avg_s = se["ms"] / n_l / 1e3
        per_launch = se["alg_bytes"] / n_l
        achieved = per_launch / avg_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak,
                "traffic": ncu_traffic(kernel_names["eval"], w.name),
                "kernel": kernel_names["eval"],
                "peak_kind": peak_kind, "alg_bytes_per_launch": per_launch,
                "avg_launch_us": avg_s * 1e6, "launches": n_l,
                "share_of_kernel_time": se["share_of_kernel_time"],
                "dominant_kernel": kernel_names[dominant]}
        if dominant != "eval":
            roof["note"] = (f"{kernel_names[dominant]} has the largest share of kernel time; it "
                            "moves no bulk data (a chain of dependent round trips per child or "
                            "slot), so the roofline is the evaluation kernel's, the path's only "
                            "bandwidth-bound kernel")
    line = {"metric": METRIC, "value": units / (total_ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-compare/int32", "data": "synthetic",
            "config": {"workload": w.name, "rows": w.rows, "cols": w.cols, "pop": w.pop,
                       "len": [w.len_lo, w.len_hi], "ratio": list(w.ratio),
                       "neg_trends": w.neg_trends, "generations": gens, "mode": args.mode,
                       "trend": args.trend,
                       "l2": "flushed between steps (512 MB write)",
                       "kernel_stats": "CUDA events around every kernel, on the library's "
                                       "stream, over a second pass of the same K steps",
                       "parallelism": f"independent job per GPU x{world}"},
            "gpu_launches": int(st_all["launches"]),
            "roofline": roof,
            "kernels": stats,
            "clocks": clk,
            "e2e": e2e}
    if gens > 0:
        line["generations_per_s"] = gens * args.steps / (total_ms / 1e3)
        line["quality"] = search_quality(ctx, truth, R, w.cols, gens)
    if not args.no_scale_roofline and w.name != "batched":
        line["roofline_at_scale"] = scale_roofline(ebic, dev, stream, peak, peak_kind)
    if not args.no_cpu_baseline:
        with OraclePool(x) as pool:
            line["cpu_baseline"] = cpu_baseline(w, x, ci, off, args.cpu_seconds, args.trend,
                                                pool=pool, generation=gens > 0)
    print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

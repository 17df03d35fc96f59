"""EBIC population-evaluation benchmark on GB300.

One step = one pass of the whole hot path over one synthetic workload, through the C ABI:
  matrix upload (order keys) -> rank codes and pair bitmap (when AUTO, as tuned, picks the
  bitmap form) -> full evaluation of the workload's population -> the EBIC generation loop
  (initial population + `--gens` generations, graph-replayed) -> bicluster extraction of the top
  list.  The metric is (individual, row) trend evaluations per second over the step; generations
  per second are reported beside it.  Default workload (the largest single-GPU one): tie-heavy,
  60,000 x 1,000 log-normal values rounded to 0.1 with 20 planted biclusters, population 8,192,
  lengths 2-64, approximate ratio 0.85, negative trends, 100 generations.  The autotuner runs
  once before the warm-up steps.  Extra keys, measured after the timed region: the exact trend on
  the same workload, the plain one-launch-per-individual form and the kernel-by-kernel loop
  against the production forms (with identical results checked), the default and batched
  workloads, the serving stream, and the CPU oracle on the host cores.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                       [--workload tieheavy|default|batched|tiny|serving] [--gens G]
                       [--mode auto|...] [--no-extras] [--no-serving] [--no-e2e]
                       [--no-cpu-baseline]
Multi-GPU (torchrun): every rank runs an independent job (its own seed) on its own GPU; the
value is all ranks' evaluations divided by the slowest rank's time ("weak" scaling).
"""

import argparse
import hashlib
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
    ap.add_argument("--workload", default="tieheavy")
    ap.add_argument("--gens", type=int, default=None, help="generations per step")
    ap.add_argument("--rows", type=int, default=0,
                    help="override the workload's rows (a smaller case of it, e.g. for profiling)")
    ap.add_argument("--cols", type=int, default=0, help="override the workload's columns")
    ap.add_argument("--pop", type=int, default=0, help="override the workload's population")
    ap.add_argument("--ipw", type=int, default=0,
                    help="individuals per work item of the staged bitmap form (0: the tuner's)")
    ap.add_argument("--fuse-pairs", type=int, default=0,
                    help="pair limit of the evaluation inside the evolve kernel (0: the library's "
                         "choice, -1: none)")
    ap.add_argument("--mode", default="auto", choices=list(MODES))
    ap.add_argument("--trend", default="strict",
                    choices=["strict", "ties", "last-kept", "ties-last-kept"],
                    help="pair test: strict (default), ties holding for both directions, "
                         "comparison with the last kept value, or both")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra keys (exact trend, vs_plain, other workloads, serving)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving extra key")
    ap.add_argument("--no-tune", action="store_true", help="AUTO without the autotuner")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed steps by cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off)")
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


def resized(w, args):
    """The workload with --rows / --cols / --pop applied (planted sizes capped to fit)."""
    import dataclasses
    rows = args.rows or w.rows
    cols = args.cols or w.cols
    pop = args.pop or w.pop
    if (rows, cols, pop) == (w.rows, w.cols, w.pop):
        return dataclasses.replace(w)
    cap = lambda r, n: (min(r[0], n), min(r[1], n))
    return dataclasses.replace(w, name=f"{w.name}-{rows}x{cols}-p{pop}", rows=rows, cols=cols,
                               pop=pop, bic_rows=cap(w.bic_rows, rows // 4),
                               bic_cols=cap(w.bic_cols, cols), len_hi=min(w.len_hi, cols))


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


# The source files each kernel with a committed traffic summary is compiled from.  A summary row
# carries a hash of them as they were when the capture ran; a row whose hash differs from the
# files now describes an earlier kernel and is not reported.
KERNEL_SOURCES = {
    "k_evolve_seq": ["evolve.cu", "tables.cuh"],
    "k_eval_bitmap": ["eval.cu", "items.cuh", "trend.cuh", "tables.cuh"],
}


def kernel_source_hash(kernel):
    """First 12 hex digits of the SHA-256 of the kernel's source files (name, NUL, contents, NUL
    each, in the listed order), or None for a kernel without a list."""
    files = KERNEL_SOURCES.get(kernel)
    if not files:
        return None
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2105_01196_gb300", "csrc", f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read() + b"\0")
    return h.hexdigest()[:12]


def ncu_traffic_entry(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu summary
    (profiles/traffic_<kernel>.txt: kernel, workload, bytes per launch, the commit whose kernel
    source the capture ran, and the hash of that source), and where it comes from; (None, None)
    when there is none, (None, why) when the row's source hash is missing or differs from the
    kernel's source files now."""
    path = os.path.join(ROOT, "profiles", "traffic_" + kernel + ".txt")
    if not os.path.exists(path):
        return None, None
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if line.startswith("#") or len(parts) < 3 or parts[:2] != [kernel, workload]:
                continue
            src = f"profiles/traffic_{kernel}.txt ({workload}"
            src += f", ncu capture of the kernel source at commit {parts[3]})" if len(parts) > 3 \
                else ")"
            now = kernel_source_hash(kernel)
            if len(parts) < 5 or now is None or parts[4] != now:
                return None, src + ": stale, the kernel's source changed since the capture"
            return float(parts[2]), src
    return None, None


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu summary, or None."""
    return ncu_traffic_entry(kernel, workload)[0]


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


def serving_measure(local, max_running, n_jobs=0, seed_offset=0):
    """The serving stream through the continuous-batching job server: every job a fresh matrix
    shape (synth.serving_stream), population 800, ratio 0.85, 50 generations.  Phase "poisson":
    jobs submitted at their Poisson arrival times (20 jobs/s); phase "saturated": every job queued
    at once.  Latency = arrival (submission) to completion; p50/p99 over the jobs."""
    import torch
    from paper_2105_01196_gb300 import ebic, synth
    cfg = synth.SERVING
    jobs, make = synth.serving_stream(n_jobs or cfg["n_jobs"], seed=cfg["seed"] + seed_offset)
    mats = [make(k) for k in range(len(jobs))]

    def params(seed):
        return ebic.Params.make(neg_trends=1, ratio_num=cfg["ratio"][0], ratio_den=cfg["ratio"][1],
                                pop_size=cfg["pop"], max_len=20, init_min_len=2, init_max_len=20,
                                n_biclusters=10, elite=10, tabu_hit_limit=0, seed=seed)
    free, _ = torch.cuda.mem_get_info(local)
    budget = int(0.6 * free)
    out = {"jobs": len(jobs), "rate_per_s": cfg["rate_per_s"], "rows": list(cfg["rows"]),
           "cols": list(cfg["cols"]), "pop": cfg["pop"], "generations": cfg["generations"],
           "shapes": "a fresh shape per job (uniform rows x cols)", "max_running": max_running,
           "hbm_budget_bytes": budget, "latency": "submission to completion"}
    for phase in ("poisson", "saturated"):
        lat = []
        evals = 0
        with ebic.Server(local, hbm_budget_bytes=budget, max_running=max_running) as srv:
            t0 = time.perf_counter()
            ids = []
            for k, (at, R, C, seed) in enumerate(jobs):
                if phase == "poisson":
                    delay = t0 + at - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                ids.append((srv.submit(mats[k], params(seed), cfg["generations"]), R))
            for jid, R in ids:
                r = srv.wait(jid)
                if r["status"] != 0:
                    raise RuntimeError(f"serving job failed: {r}")
                lat.append(r["queued_ms"] + r["run_ms"])
                evals += r["n_evaluated"] * R
            wall = time.perf_counter() - t0
        out[phase] = {"jobs_per_s": len(jobs) / wall, "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)), "wall_s": wall,
                      "evals_per_s": evals / wall}
    return out


def run_serving(args, world, rank, local, dist):
    """`--workload serving`: the serving stream alone, as its own JSON line."""
    import torch
    torch.cuda.set_device(local)
    out = serving_measure(local, args.max_running, args.jobs, 7919 * rank)
    if rank == 0:
        line = {"metric": "EBIC jobs/sec and p50/p99 job latency (continuous batching)",
                "value": out["saturated"]["jobs_per_s"], "unit": "jobs/s", "n_gpus": world,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32-compare/int32", "data": "synthetic",
                "config": {"workload": "serving", **{k: v for k, v in out.items()
                                                    if k not in ("poisson", "saturated")}},
                "poisson": out["poisson"], "saturated": out["saturated"]}
        print(json.dumps(line), flush=True)


class Job:
    """One workload on one context: device inputs, pinned host copies, and one step of the hot
    path (upload -> evaluation sweep -> initial population + generations -> extraction)."""

    def __init__(self, ebic, torch, w, dev, stream, mode, trend, gens, host_copies=True, ipw=0,
                 fuse_pairs=0):
        self.ebic, self.torch, self.w, self.gens = ebic, torch, w, gens
        self.x, self.truth, self.ci, self.off = synth_inputs(w)
        self.R, self.P = w.rows, len(self.off) - 1
        self.x_d = torch.from_numpy(self.x).to(dev)
        self.ci_d = torch.from_numpy(self.ci).to(dev)
        self.off_d = torch.from_numpy(self.off).to(dev)
        self.outs_d = [torch.zeros(self.P, dtype=torch.int32, device=dev) for _ in range(3)]
        self.outs_d.append(torch.zeros(self.P, dtype=torch.int64, device=dev))
        if host_copies:
            # (every input the end-to-end step copies comes from pinned host memory)
            self.x_h = torch.from_numpy(self.x).pin_memory()
            self.ci_h = torch.from_numpy(self.ci).pin_memory()
            self.off_h = torch.from_numpy(self.off).pin_memory()
            self.outs_h = [torch.zeros(self.P, dtype=torch.int32).pin_memory() for _ in range(3)]
            self.outs_h.append(torch.zeros(self.P, dtype=torch.int64).pin_memory())
        self.params = ebic.Params.make(mode=MODES[mode], ipw=ipw, fuse_pairs=fuse_pairs,
                                       **run_fields(w, trend))
        self.ctx = ebic.Context(dev.index or 0, stream.cuda_stream)
        self.used_mode = 0

    def tune(self):
        """The autotuner on this matrix and population, for the step's expected sweeps (the
        evaluation sweep, the initial population and every generation); AUTO then follows it."""
        self.ctx.load_matrix(self.x_d)
        return self.ctx.autotune(self.ci_d, self.off_d, self.params, self.gens + 2)

    def step(self, host=False, around_sweep=None):
        """One pass of the hot path; returns the (individual, row) evaluations done.
        around_sweep(0 | 1), when given, is called right before and after the evaluation sweep."""
        ctx = self.ctx
        if host:
            ctx.load_matrix(self.x_h)
            ctx.eval_population(self.ci_h, self.off_h, self.params, *self.outs_h)
        else:
            ctx.load_matrix(self.x_d)
            if around_sweep:
                around_sweep(0)
            ctx.eval_population(self.ci_d, self.off_d, self.params, *self.outs_d)
            if around_sweep:
                around_sweep(1)
        units = self.P * self.R
        if self.gens > 0:
            rep = ctx.run_generations(self.params, self.gens)
            self.used_mode = int(rep.eval_mode)
            units += int(rep.n_evaluated) * self.R
            units += len(ctx.extract_biclusters(self.R)) * self.R
        return units

    def params_ratio(self):
        return self.params.ratio_num, self.params.ratio_den

    def close(self):
        self.ctx.close()


_INPUTS = {}


def synth_inputs(w):
    from paper_2105_01196_gb300 import synth
    key = (w.name, w.seed)
    if key not in _INPUTS:
        _INPUTS[key] = synth.workload_inputs(w)
    return _INPUTS[key]


def timed_steps(job, stream, flush, steps, dist=None, profile_range=False):
    """`steps` steps, each from a flushed L2 (the flush outside the events), CUDA events on the
    library's stream; returns (total ms, units).  profile_range: the steps are bracketed by
    cudaProfilerStart / Stop, so that `ncu --profile-from-start off` captures only their
    launches."""
    torch = job.torch
    total_ms, units = 0.0, 0
    if profile_range:
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        units += job.step(False)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    if profile_range:
        torch.cuda.profiler.stop()
    return total_ms, units


def kernel_stats(job, stream, flush, steps):
    """A second pass of the same steps with CUDA events around every kernel of the path (event
    nodes inside the generation graphs): per-kernel durations, work and shares, and the pass's
    own time per step (the event nodes keep consecutive kernels from overlapping).  The
    evaluation kernel's launches are also split into the step's one full sweep ("eval_sweep")
    and the generation loop's ("eval_loop")."""
    ebic, torch, ctx = job.ebic, job.torch, job.ctx
    ctx.profile_enable(True)
    sweep = {"launches": 0, "timed_launches": 0, "ms": 0.0, "alg_bytes": 0.0}
    mark = {}

    def around(k):
        st = ctx.profile_read(ebic.KERNEL_EVAL)   # (synchronises: the sweep's events are done)
        if k == 0:
            mark.update(st)
        else:
            for key in sweep:
                sweep[key] += st[key] - mark[key]
    total_ms = 0.0
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        job.step(False, around_sweep=around)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    ms = total_ms
    stats = {name: ctx.profile_read(kid) for name, kid in
             (("eval", ebic.KERNEL_EVAL), ("evolve", ebic.KERNEL_EVOLVE),
              ("finish", ebic.KERNEL_FINISH), ("bitmap_build", ebic.KERNEL_BITMAP_BUILD),
              ("rank_codes", ebic.KERNEL_RANK_CODES))}
    ctx.profile_enable(False)
    ev = stats["eval"]
    stats["eval_sweep"] = dict(sweep)
    stats["eval_loop"] = {key: ev[key] - sweep[key] for key in sweep}
    tot = sum(v["ms"] for k, v in stats.items() if k not in ("eval_sweep", "eval_loop"))
    for v in stats.values():
        v["avg_us"] = 1e3 * v["ms"] / v["timed_launches"] if v["timed_launches"] else None
        v["share_of_kernel_time"] = v["ms"] / tot if tot else None
    return stats, {"instrumented_ms_per_step": ms / steps, "kernel_ms_per_step": tot / steps}


def eval_roofline(stats, kernel, peak, peak_kind, traffic, traffic_source, part="eval"):
    se = stats[part]
    if not (se["timed_launches"] > 0 and se["ms"] > 0):
        return None
    n_l = se["timed_launches"]
    avg_s = se["ms"] / n_l / 1e3
    per_launch = se["alg_bytes"] / n_l
    achieved = per_launch / avg_s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "traffic_source": traffic_source,
            "kernel": kernel, "peak_kind": peak_kind, "alg_bytes_per_launch": per_launch,
            "avg_launch_us": avg_s * 1e6, "launches": n_l,
            "share_of_kernel_time": se["share_of_kernel_time"]}


def workload_summary(job, stream, flush, steps, warmup, peak, peak_kind):
    """A workload's step rate, generations/s and evaluation-kernel roofline (outside the headline's
    timed region)."""
    job.tune()
    for _ in range(warmup):
        job.step(False)
    ms, units = timed_steps(job, stream, flush, steps)
    stats, passes = kernel_stats(job, stream, flush, steps)
    w = job.w
    out = {"value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
           "steps": steps, "rows": w.rows, "cols": w.cols, "pop": w.pop,
           "len": [w.len_lo, w.len_hi], "ratio": list(job.params_ratio()),
           "generations": job.gens, "eval_form": eval_kernel_name(job.used_mode, w.cols),
           "roofline": eval_roofline(stats, eval_kernel_name(job.used_mode, w.cols), peak,
                                     peak_kind,
                                     *ncu_traffic_entry(eval_kernel_name(job.used_mode, w.cols),
                                                        w.name + ("-loop" if job.gens > 0
                                                                  else "")),
                                     "eval_loop" if job.gens > 0 else "eval"),
           "kernel_ms": {k: v["ms"] / steps for k, v in stats.items()}, **passes}
    if job.gens > 0:
        out["generations_per_s"] = job.gens * steps / (ms / 1e3)
    return out


def vs_plain(job, stream, gens_loop=20):
    """The target's comparison, on the headline workload: (1) one evaluation sweep of the
    population in the paper's form (EBIC_MODE_PLAIN, one launch per individual) against the
    production form (AUTO, as tuned), with equal counts and fitness checked; (2) the generation
    loop launched kernel by kernel (use_graph = 0, the host reading the progress counters every
    generation) against the graph-replayed loop, with equal top lists and populations checked."""
    ebic, torch, ctx = job.ebic, job.torch, job.ctx
    P = job.P
    ctx.load_matrix(job.x_d)
    res = {}
    outs = {}
    for name, mode in (("plain", MODES["plain"]), ("batched", MODES["auto"])):
        p = ebic.Params.make(mode=mode, **run_fields(job.w))
        o = [torch.zeros(P, dtype=torch.int32, device=job.x_d.device) for _ in range(3)]
        o.append(torch.zeros(P, dtype=torch.int64, device=job.x_d.device))
        ctx.eval_population(job.ci_d, job.off_d, p, *o)                # warm-up (and build)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.eval_population(job.ci_d, job.off_d, p, *o)
        e1.record(stream)
        e1.synchronize()
        res[name + "_sweep_ms"] = e0.elapsed_time(e1)
        outs[name] = [t.cpu().numpy() for t in o]
    sweep_same = all(np.array_equal(a, b) for a, b in zip(outs["plain"], outs["batched"]))
    loop = {}
    for name, graph in (("eager", 0), ("graph", 1)):
        p = ebic.Params.make(mode=MODES["auto"], use_graph=graph, **run_fields(job.w))
        ctx.load_matrix(job.x_d)
        ctx.run_generations(p, 0)                                       # initial population
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep = ctx.run_generations(p, gens_loop)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        pop = ctx.population(P)
        loop[name] = {"ms_per_generation": 1e3 * dt / gens_loop, "gens_done": rep.gens_done,
                      "top": [(e["cols"], e["f"]) for e in ctx.toplist()],
                      "pop": [np.asarray(a).tolist() for a in pop]}
    loop_same = (loop["eager"]["top"] == loop["graph"]["top"]
                 and loop["eager"]["pop"] == loop["graph"]["pop"]
                 and loop["eager"]["gens_done"] == loop["graph"]["gens_done"] == gens_loop)
    return {"sweep": {"plain_ms": res["plain_sweep_ms"], "batched_ms": res["batched_sweep_ms"],
                      "speedup": res["plain_sweep_ms"] / res["batched_sweep_ms"],
                      "plain_launches": P, "identical": bool(sweep_same)},
            "loop": {"generations": gens_loop,
                     "eager_ms_per_generation": loop["eager"]["ms_per_generation"],
                     "graph_ms_per_generation": loop["graph"]["ms_per_generation"],
                     "speedup": loop["eager"]["ms_per_generation"]
                     / loop["graph"]["ms_per_generation"],
                     "identical": bool(loop_same)},
            "identical": bool(sweep_same and loop_same),
            "timing": "sweep: CUDA events on the library stream; loop: host clock around the "
                      "call, device synchronised on both sides"}


def quality_variants(ebic, torch, dev, stream):
    """Clustering error (Eq. 1) of a 100-generation run on the default workload (10,000 x 100,
    P 800) under the paper's trend parameters: negative trends on or off, approximate ratio 0.85
    or the exact trend (no reading of the method changes between them)."""
    import dataclasses
    from paper_2105_01196_gb300 import synth
    w0 = synth.WORKLOADS["default"]
    out = []
    for neg, ratio in ((1, (85, 100)), (0, (85, 100)), (1, (1, 1)), (0, (1, 1))):
        w = dataclasses.replace(w0, neg_trends=neg, ratio=ratio)
        job = Job(ebic, torch, w, dev, stream, "auto", "strict", w.generations, host_copies=False)
        job.step(False)
        q = search_quality(job.ctx, job.truth, job.R, w.cols, w.generations)
        out.append({"neg_trends": neg, "ratio": list(ratio), "ce_score": q["ce_score"],
                    "best_pair_score_per_planted": q["best_pair_score_per_planted"]})
        job.close()
    return out


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
    w = resized(synth.WORKLOADS[args.workload], args)
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
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peak, peak_kind = load_peaks()

    job = Job(ebic, torch, w, dev, stream, args.mode, args.trend, gens, ipw=args.ipw,
              fuse_pairs=args.fuse_pairs)
    tune = job.tune() if args.mode == "auto" and not args.no_tune else None
    for _ in range(max(3, args.warmup)):
        job.step(False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    job.ctx.profile_enable(True)        # reset the launch counters ...
    job.ctx.profile_enable(False)       # ... and time this pass without per-kernel events
    total_ms, units = timed_steps(job, stream, flush, args.steps,
                                  profile_range=args.profile_range)
    st_all = job.ctx.profile_read(ebic.KERNEL_ALL)
    clk = clocks.stop()
    stats, passes = kernel_stats(job, stream, flush, args.steps)
    if dist:
        total_ms, units = reduce_over_ranks(dist, total_ms, units, dev)

    e2e = None
    if not args.no_e2e:
        # End to end through the same C ABI with host buffers: the copies run inside the calls.
        # Each step is timed on the host clock from a flushed L2, like the device-timed steps.
        e2e_units, e2e_s = 0, 0.0
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_units += job.step(True)
            torch.cuda.synchronize()
            e2e_s += time.perf_counter() - t0
        h2d = job.x.nbytes + job.ci.nbytes + job.off.nbytes
        d2h = sum(o.numel() * o.element_size() for o in job.outs_h)
        if gens > 0:
            d2h += 256 * ((job.R + 127) // 128) * 16
        e2e = {"value": e2e_units / e2e_s * (world if dist else 1), "unit": UNIT,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    if rank != 0:
        job.close()
        if dist:
            dist.destroy_process_group()
        return

    eval_name = eval_kernel_name(job.used_mode if job.used_mode else MODES[args.mode], w.cols)
    # (the library's choice: a warp per slot once the slots' attempt warps exceed the GPU's)
    g_att = 1
    while g_att < job.params.max_attempts:
        g_att *= 2
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    evolve_name = "k_evolve_seq" if job.P * g_att > sms * 32 else "k_evolve"
    names = {"eval": eval_name, "evolve": evolve_name, "finish": "k_finish",
             "bitmap_build": "k_build_bitmap_planes" if w.cols <= 1024 else "k_build_bitmap",
             "rank_codes": "k_rank_codes"}
    dominant = max((k for k in stats if k not in ("eval_sweep", "eval_loop")),
                   key=lambda k: stats[k]["ms"])
    loop_tag = w.name + ("-loop" if gens > 0 else "")
    # The generation loop's evaluations: with the bitmap form the evolve kernel scores its short
    # exact children itself (the pair words it reads are its algorithmic bytes) and the
    # evaluation launches score the rest.  The roofline is the kernel with the larger share of
    # the two, the other one and the step's one full sweep beside it.
    part = "eval_loop" if gens > 0 else "eval"
    roof_eval = eval_roofline(stats, eval_name, peak, peak_kind,
                              *ncu_traffic_entry(eval_name, loop_tag), part)
    roof_evolve = None
    if gens > 0 and stats["evolve"]["alg_bytes"] > 0:
        roof_evolve = eval_roofline(stats, evolve_name, peak, peak_kind,
                                    *ncu_traffic_entry("k_evolve_seq", loop_tag), "evolve")
    if roof_evolve is not None and stats["evolve"]["ms"] >= stats["eval_loop"]["ms"]:
        roof = roof_evolve
        roof["launches_measured"] = ("the generation loop's evolve launches; their algorithmic "
                                     "bytes are the pair words (and pair counts) of the children "
                                     "they evaluate; they also build every child (dependent "
                                     "loads, no bulk data)")
        roof["eval_launches"] = roof_eval
    else:
        roof = roof_eval
        if roof is not None and gens > 0:
            roof["launches_measured"] = ("the generation loop's evaluation launches (initial "
                                         "population and every generation)")
            if roof_evolve is not None:
                roof["evolve_launches"] = roof_evolve
    if roof is not None and gens > 0:
        roof["sweep"] = eval_roofline(stats, eval_name, peak, peak_kind,
                                      *ncu_traffic_entry(eval_name, w.name), part="eval_sweep")
    if roof is not None:
        roof["dominant_kernel"] = names[dominant]
        if dominant not in ("eval", "evolve"):
            roof["note"] = (f"{names[dominant]} has the largest share of kernel time; it moves "
                            "no bulk data, so the roofline is the evaluation's")
    line = {"metric": METRIC, "value": units / (total_ms / 1e3), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32-compare/int32", "data": "synthetic",
            "config": {"workload": w.name, "rows": w.rows, "cols": w.cols, "pop": w.pop,
                       "len": [w.len_lo, w.len_hi], "ratio": list(w.ratio),
                       "neg_trends": w.neg_trends, "generations": gens, "mode": args.mode,
                       "trend": args.trend,
                       "l2": "flushed between steps (512 MB write); the pair bitmap (7.5 GB "
                             "at 60,000 x 1,000) is larger than L2 too",
                       "kernel_stats": "CUDA events around every kernel, on the library's "
                                       "stream, over a second pass of the same K steps",
                       "parallelism": f"independent job per GPU x{world}"},
            "gpu_launches": int(st_all["launches"]),
            "roofline": roof,
            "kernels": stats,
            "kernel_passes": dict(passes, timed_ms_per_step=total_ms / args.steps),
            "clocks": clk,
            "e2e": e2e}
    if tune is not None:
        line["config"]["autotune"] = {k: tune[k] for k in ("mode", "seg_direct", "seg_bitmap",
                                                          "seg_loop", "ipw_bitmap", "ipw_loop",
                                                          "fuse_loop",
                                                          "direct_ms", "bitmap_ms", "build_ms",
                                                          "staged_ms")}
    if gens > 0:
        line["generations_per_s"] = gens * args.steps / (total_ms / 1e3)
        line["quality"] = search_quality(job.ctx, job.truth, job.R, w.cols, gens)
    if not args.no_extras:
        # (outside the headline's timed region)
        if w.ratio != (1, 1):
            ex = Job(ebic, torch, dataclasses.replace(w, ratio=(1, 1)), dev, stream, args.mode,
                     args.trend, gens, host_copies=False)
            line["exact_trend"] = workload_summary(ex, stream, flush, args.steps, 3, peak,
                                                   peak_kind)
            ex.close()
        line["vs_plain"] = vs_plain(job, stream)
        line["workloads"] = {}
        for name in ("default", "batched"):
            if name == w.name:
                continue
            wo = synth.WORKLOADS[name]
            jo = Job(ebic, torch, wo, dev, stream, args.mode, args.trend, wo.generations,
                     host_copies=False)
            line["workloads"][name] = workload_summary(jo, stream, flush, args.steps, 3, peak,
                                                       peak_kind)
            jo.close()
        line["quality_default_workload"] = quality_variants(ebic, torch, dev, stream)
        if not args.no_serving:
            line["serving"] = serving_measure(local, args.max_running, args.jobs)
    if not args.no_cpu_baseline:
        with OraclePool(job.x) as pool:
            line["cpu_baseline"] = cpu_baseline(w, job.x, job.ci, job.off, args.cpu_seconds,
                                                args.trend, pool=pool, generation=gens > 0)
    print(json.dumps(line), flush=True)
    job.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Benchmark of the Hypercurves hot path on GB300.

One step = the whole path over one batch of synthetic input, with the inputs
already resident in HBM:
  hc_build  Algorithm 1: Hilbert keys of N rows x 8 curves + radix sort
  hc_query  Algorithm 2 for Q queries: keys, lower_bound, window gathers,
            exact distances, top-k merged over curves
value = queries answered per second of step time (whole job, all ranks).

Workload (default): N = 10,000,000 uint8 rows of 128 dims from the seeded
64-cluster Gaussian mixture (sigma 20) standing in for SIFT, Q = 100,000
queries (rows + N(0, 8)), 8 curves of 16 dims, p = 128 per side, k = 10.
The database (1.28 GB) and the index (1.6 GB) are larger than L2, so no L2
flush is needed between steps.

`--impl reference` times the CPU oracle instead (the reference arm: a
deliberately plain program) on the whole job of every step.

Multi-GPU: one process per GPU under torchrun; every rank runs an
independent replica (its own index and query batch), with no collective on
the data path (weak scaling); only the step timings are reduced (max).
"""
import argparse
import collections
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("queries/s at fixed recall@10, 10M×128-d uint8, 8 curves; % HBM peak; "
          "p99 latency")
UNIT = "queries/s"
DATA = ("synthetic: seeded 64-cluster isotropic Gaussian mixture (centres uniform in "
        "[0,255], sigma 20, rounded and clipped) standing in for 128-d SIFT; queries are "
        "database rows plus N(0, 8) noise")
QUERY_SOURCES = ["paper_1209_0410_gb300/csrc/query.cu", "paper_1209_0410_gb300/csrc/hc_topk.cuh",
                 "paper_1209_0410_gb300/csrc/hc_device.cuh",
                 "paper_1209_0410_gb300/csrc/hc_query_dev.cuh"]


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["hc", "reference"], default="hc")
    ap.add_argument("--e2e-depth", type=int, default=2,
                    help="end-to-end line: databases uploaded ahead of the step being answered")
    ap.add_argument("--workload", choices=["scale", "uneven", "learned", "serve", "partitions"],
                    default="scale",
                    help="scale: the headline (build + query at N=10M); uneven: 64 indexes in "
                         "one persistent launch; learned: learned probe depth; serve: online "
                         "serving under fluctuating load; partitions: partitioned "
                         "Hypercurves, Optimist/Pessimist slack")
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    ap.add_argument("--serve-n", type=int, default=50_000_000)
    ap.add_argument("--train-queries", type=int, default=1_000_000)
    ap.add_argument("--heldout-queries", type=int, default=100_000)
    ap.add_argument("--tune-cache", default=None, help="autotuner JSON cache path")
    ap.add_argument("--n-db", type=int, default=10_000_000)
    ap.add_argument("--nq", type=int, default=100_000)
    ap.add_argument("--p", type=int, default=128)
    ap.add_argument("--k", type=int, default=10)
    ap.add_argument("--dtype", choices=["u8", "f32"], default="u8")
    ap.add_argument("--sweep", default="32,64,128,256,512",
                    help="query-only p sweep ('' = none)")
    ap.add_argument("--recall-sample", type=int, default=2000)
    ap.add_argument("--input-order", action="store_true",
                    help="answer the queries in input order (hc_query) instead of curve-0 key "
                         "order (hc_query_ordered)")
    ap.add_argument("--quick", action="store_true",
                    help="timed steps only: no sweep, recall, e2e or CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-queries", type=int, default=4000,
                    help="queries of the oracle's bounded search sample (CPU baseline)")
    return ap.parse_args()


# ----------------------------------------------------------------- helpers
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms, world, device):
    """The timed region's length on the slowest rank (ms).  The only collective
    of the benchmark: the ranks' query batches are independent, so nothing is
    exchanged on the data path."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ms_per_step, nq_per_rank, world):
    """Whole-job queries/s: every rank answers its own nq queries per step
    (weak scaling), and the step lasts as long as the slowest rank's."""
    return world * nq_per_rank / (ms_per_step / 1000.0)


def workload_name(a):
    return ("plain Hypercurves at scale: N=%d x %d-d %s, 8 curves x 16 dims, Q=%d, p=%d, k=%d; "
            "step = index build + query batch" % (a.n_db, 128, "uint8" if a.dtype == "u8"
                                                   else "float32 (u8/255)", a.nq, a.p, a.k))


def make_inputs(a, rank):
    import numpy as np
    from paper_1209_0410_gb300 import datagen
    db = datagen.make_db(a.n_db, 128, seed=datagen.SEED_DB)
    q = datagen.make_queries(db, a.nq, seed=datagen.SEED_QUERIES + 1000 * rank)
    if a.dtype == "f32":
        db, q = datagen.to_f32(db), datagen.to_f32(q)
    return np.ascontiguousarray(db), np.ascontiguousarray(q)


def source_sha(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def ncu_traffic(kernel_tag):
    """Per-launch DRAM bytes from the committed ncu summary of this kernel, if
    the summary was taken on the current source (else None)."""
    path = os.path.join(ROOT, "profiles", "%s.md" % kernel_tag)
    if not os.path.exists(path):
        return None, None
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha") != source_sha(QUERY_SOURCES):
        return None, vals.get("source_sha")
    try:
        return float(vals["dram_bytes_per_launch"]), vals.get("source_sha")
    except (KeyError, ValueError):
        return None, vals.get("source_sha")


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
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
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu),
                                          "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, st in rows for i, v in enumerate(st)
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


BUILD_PASSES = 6   # radix passes of a 16-coordinate build: the top 6 bytes of the high word
E2E_RUNS = 5       # timed runs of the end-to-end pipeline; the line reports their median


def build_bytes(n, row_bytes, curves, passes=BUILD_PASSES):
    """Bytes of one index build of n rows and `curves` lists.

    algorithmic: the method's own traffic, counted by record -- the rows
    read once, c n (key, id) records of 20 bytes written, and every radix pass
    reading and writing every record.
    kernel: what the build's kernels move -- the key pass (rows in, 8-byte high
    words and the first pass's digit byte out); per pass the histogram (one
    digit byte per record), the digit counts (written, scanned, read back: one 4-byte
    word per digit and 4096-record tile, four times), and the scatter (word
    and position in -- the first pass derives positions -- word and position
    out plus the next pass's digit byte; the last pass writes ids in place of
    positions and no digit); then the run fix-up's read of the high words and
    ids (it reorders the short runs in place; the few records it moves are
    not counted) and its write of the search fence (every 16th high word)."""
    r = curves * n
    algorithmic = n * row_bytes + r * 20 + passes * 2 * r * 20
    counts = 4 * 4 * 256 * (r / 4096.0)
    kernel = n * row_bytes + r * 9                      # key pass: words + first digits
    for t in range(passes):
        first, last = t == 0, t == passes - 1
        kernel += r * 1 + counts                        # histogram + counts
        kernel += r * (8 if first else 12)              # scatter reads
        kernel += r * (12 if last else 13)              # scatter writes
    kernel += r * 12                                    # run fix-up
    kernel += r * 0.5                                   # fence: 8 B per 16 entries
    return float(algorithmic), float(kernel)


def algorithmic_query_bytes(hc, idx, q_dev, p, k, row_bytes):
    """Bytes the method itself must move for one query launch (per query:
    window ids 4 B + window rows, every probe of the binary search in every
    list at 8 B (the high key word; the low word is needed only on the rare
    ties; the kernel stages no levels in shared memory), the query row and k
    (id, distance) results)."""
    import torch
    pos = hc.hc_query_positions(idx, q_dev)
    _, off = hc.hc_index_describe(idx)
    n_list = torch.tensor((off[1:] - off[:-1]).astype("int64"), device=pos.device)
    lo = torch.clamp(pos - p, min=0)
    hi = torch.minimum(pos + p, n_list.unsqueeze(0))
    windows = int((hi - lo).clamp(min=0).sum().item())
    nq, lists = pos.shape
    lg = sum(int(n).bit_length() for n in (off[1:] - off[:-1]).tolist())
    return windows * (row_bytes + 4) + nq * (lg * 8 + row_bytes + k * 8), windows


def recall_at_10(ids, dist, true_dist):
    import torch
    kth = true_dist[:, 9:10].to(torch.float64)
    ok = (dist[:, :10].to(torch.float64) <= kth) & (ids[:, :10] >= 0)
    return float(ok.sum(dim=1).clamp(max=10).to(torch.float64).mean().item() / 10.0)


def fixed_recall_point(sweep, ref_p):
    """The smallest swept depth whose recall@10 reaches the recall at ref_p (the
    metric's fixed recall), with its query throughput; None without ref_p."""
    ref = [e for e in sweep if e["p"] == ref_p]
    if not ref:
        return None
    target = ref[0]["recall_at_10"]
    best = min((e for e in sweep if e["recall_at_10"] >= target), key=lambda e: e["p"])
    return {"p": best["p"], "recall_at_10": best["recall_at_10"],
            "target_recall_at_10": target, "query_qps": best["query_qps"]}


# ----------------------------------------------------------- CPU oracle leg
def cpu_oracle_sample(a, db, q):
    """Times the oracle (as it stands) on the machine's host cores: the build of
    the whole index (all N rows, unscaled) plus the search of a bounded
    sample of the queries, scaled to Q (queries are answered independently).
    A single-core figure (the setting of the paper's speedups) comes from a
    tenth of the rows, scaled by n log n, and a small query sample."""
    from oracle import oracle as O
    threads = os.cpu_count() or 1
    nqs = min(a.cpu_queries, a.nq)
    t0 = time.perf_counter()
    oidx = O.build(db, curves=8, m=16, nthreads=threads)
    t1 = time.perf_counter()
    O.search(oidx, db, q[:nqs], a.k, a.p, nthreads=threads)
    t2 = time.perf_counter()
    del oidx
    t_job = (t1 - t0) + (t2 - t1) * (a.nq / nqs)
    r1, q1 = max(2, a.n_db // 10), max(1, nqs // 20)
    t3 = time.perf_counter()
    oidx1 = O.build(db[:r1], curves=8, m=16, nthreads=1)
    t4 = time.perf_counter()
    O.search(oidx1, db[:r1], q[:q1], a.k, a.p, nthreads=1)
    t5 = time.perf_counter()
    del oidx1
    nlogn = (a.n_db * math.log2(a.n_db)) / (r1 * math.log2(r1))
    t_job1 = (t4 - t3) * nlogn + (t5 - t4) * (a.nq / q1)
    return {"value": a.nq / t_job, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": ("oracle build of all %d rows (8 lists, %.2f s, unscaled) + search of %d "
                       "of the %d queries at p=%d on %d threads (%.2f s, scaled x%.1f); "
                       "whole-job time %.2f s"
                       % (a.n_db, t1 - t0, nqs, a.nq, a.p, threads, t2 - t1, a.nq / nqs,
                          t_job)),
            "build_s": t1 - t0,
            "single_core": {"value": a.nq / t_job1, "unit": UNIT, "cores": 1,
                            "sample": "build of %d rows (%.2f s, scaled by n log n to N) + "
                                      "search of %d queries (scaled to Q), one thread"
                                      % (r1, t4 - t3, q1)}}


def run_reference(a):
    """The reference arm: the CPU oracle on the whole job of every step (the
    index build over all N rows plus the search of all Q queries, on the
    host's cores), nothing scaled."""
    from oracle import oracle as O
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    db, q = make_inputs(a, 0)
    threads = os.cpu_count() or 1

    def step(frac=1):
        n, nq = a.n_db // frac, a.nq // frac
        oidx = O.build(db[:n], curves=8, m=16, nthreads=threads)
        O.search(oidx, db[:n], q[:nq], a.k, a.p, nthreads=threads)

    # untimed warm-up steps run the same code on a tenth of the job, so that
    # the whole run stays within a few minutes; every timed step is whole
    for _ in range(a.warmup):
        step(10)
    times = []
    t_run = time.perf_counter()
    for _ in range(a.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    t_run = time.perf_counter() - t_run
    t_step = statistics.mean(times)
    value = a.nq / t_step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": t_step * 1000.0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": a.dtype, "data": DATA,
            "config": {"workload": workload_name(a), "n_db": a.n_db, "nq": a.nq, "p": a.p,
                       "k": a.k, "curves": 8, "dims_per_curve": 16,
                       "timed_region_s": t_run,
                       "note": "every timed step is the whole job on the CPU oracle: the "
                               "build of all N rows and the search of all Q queries, "
                               "unscaled (untimed warm-up steps run a tenth of it)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": "the whole job (all %d rows, all %d queries) per step, "
                                       "%d timed steps, unscaled" % (a.n_db, a.nq, a.steps)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ GPU leg
def run_hc(a):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_1209_0410_gb300 import hc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    hc.lib()
    db_np, q_np = make_inputs(a, rank)
    row_bytes = 128 * (4 if a.dtype == "f32" else 1)
    db = torch.from_numpy(db_np).cuda()
    q = torch.from_numpy(q_np).cuda()
    stream = torch.cuda.current_stream()
    out_ids = torch.empty((a.nq, a.k), dtype=torch.int32, device="cuda")
    out_dist = torch.empty((a.nq, a.k), dtype=torch.float32 if a.dtype == "f32" else torch.int32,
                           device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()

    workspace = []   # sized by the first index (every step's index has the same lists)

    def query(idx, p=None):
        if a.input_order:
            hc.hc_query(idx, q, a.k, a.p if p is None else p, out_ids, out_dist, stream=stream)
        else:
            if not workspace:
                workspace.append(torch.empty(hc.hc_query_ordered_workspace(idx, a.nq),
                                             dtype=torch.uint8, device="cuda"))
            hc.hc_query_ordered(idx, q, a.k, a.p if p is None else p, out_ids, out_dist,
                                workspace=workspace[0], stream=stream)

    def step(ev):
        ev[0].record(stream)
        idx = hc.hc_build(db, 8, 16, stream=stream)
        ev[1].record(stream)
        query(idx)
        ev[2].record(stream)
        idx.free(stream=stream)

    mk = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for _ in range(a.warmup):
        step(mk())
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
    events = [mk() for _ in range(a.steps)]
    barrier()
    torch.cuda.synchronize()
    launches0 = hc.hc_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for i in range(a.steps):
        step(events[i])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = hc.hc_launch_count() - launches0
    clocks = sampler.stop() if rank == 0 else None

    total_ms = t_start.elapsed_time(t_end)
    build_ms = [e[0].elapsed_time(e[1]) for e in events]
    query_ms = [e[1].elapsed_time(e[2]) for e in events]
    step_ms = [e[0].elapsed_time(e[2]) for e in events]
    ms_per_step = max_over_ranks(total_ms, world, "cuda") / a.steps
    value = job_throughput(ms_per_step, a.nq, world)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    idx = hc.hc_build(db, 8, 16, stream=stream)
    torch.cuda.synchronize()
    qbytes, windows = algorithmic_query_bytes(hc, idx, q, a.p, a.k, row_bytes)
    q_ms = statistics.mean(query_ms)
    peaks, peak_src = measured_peaks()
    achieved = qbytes / (q_ms / 1000.0) / 1e9
    # the committed capture is of the default workload only
    traffic, _ = ncu_traffic("query_kernel")
    if (a.n_db, a.nq, a.p, a.k, a.dtype, a.input_order) != (10_000_000, 100_000, 128, 10, "u8",
                                                            False):
        traffic = None
    roofline = {"kernel": "hc_query_ordered: order keys + sort + batch lower_bound (K1, K3) "
                          "+ query_kernel walk (K4..K6); time of the whole call",
                "bound": "hbm",
                "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"],
                "traffic": traffic,
                "algorithmic_bytes_per_launch": qbytes,
                # DRAM bytes of the launch (ncu) over its duration: below `frac` when
                # window rows are shared in L2 by queries answered together
                "dram_frac": (traffic / (q_ms / 1000.0) / 1e9 / peaks["hbm_gbs"]
                              if traffic else None),
                "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_src
                if peak_src == "measured" else "fallback 6.8 TB/s"}

    b_ms = statistics.mean(build_ms)
    alg_b, ker_b = build_bytes(a.n_db, row_bytes, 8)
    roofline_build = {"kernels": "build_keys + %d x (hist, scan, scatter) + run fix-up"
                                 % BUILD_PASSES,
                      "bound": "hbm", "unit": "GB/s", "peak": peaks["hbm_gbs"],
                      "ms": b_ms, "algorithmic_bytes": alg_b, "kernel_bytes": ker_b,
                      "achieved": alg_b / (b_ms / 1000.0) / 1e9,
                      "frac": alg_b / (b_ms / 1000.0) / 1e9 / peaks["hbm_gbs"],
                      "kernel_achieved": ker_b / (b_ms / 1000.0) / 1e9,
                      "kernel_frac": ker_b / (b_ms / 1000.0) / 1e9 / peaks["hbm_gbs"]}

    cfg = {"workload": workload_name(a), "n_db": a.n_db, "nq": a.nq, "p": a.p, "k": a.k,
           "curves": 8, "dims_per_curve": 16, "partitions": 1,
           "query_order": ("input order (hc_query)" if a.input_order else
                           "curve-0 key order (hc_query_ordered; results identical)"),
           "l2": "inputs larger than L2 (database %.2f GB, index %.2f GB vs 129 MB L2)"
                 % (a.n_db * row_bytes / 1e9, a.n_db * 8 * 12 / 1e9),
           "build_ms": statistics.mean(build_ms), "query_ms": q_ms,
           "query_only_qps": a.nq / (q_ms / 1000.0),
           "step_latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                               "p99": float(np.percentile(step_ms, 99))},
           "window_rows_per_query": windows / a.nq}

    if not a.quick and a.recall_sample > 0:
        rs = min(a.recall_sample, a.nq)
        tids, tdist = hc.hc_bruteforce(db, q[:rs], 10)
        torch.cuda.synchronize()
        cfg["recall_at_10"] = recall_at_10(out_ids[:rs], out_dist[:rs], tdist)
        cfg["recall_sample_queries"] = rs
        sweep = []
        for p in [int(x) for x in a.sweep.split(",") if x.strip()]:
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            query(idx, p)
            ev[0].record(stream)
            reps = 3
            for _ in range(reps):
                query(idx, p)
            ev[1].record(stream)
            torch.cuda.synchronize()
            ms = ev[0].elapsed_time(ev[1]) / reps
            qb, _ = algorithmic_query_bytes(hc, idx, q, p, a.k, row_bytes)
            sweep.append({"p": p, "query_ms": ms, "query_qps": a.nq / (ms / 1000.0),
                          "recall_at_10": recall_at_10(out_ids[:rs], out_dist[:rs], tdist),
                          "hbm_frac": qb / (ms / 1000.0) / 1e9 / peaks["hbm_gbs"]})
        cfg["query_sweep"] = sweep
        cfg["fixed_recall_point"] = fixed_recall_point(sweep, a.p)
    idx.free()

    e2e = None
    if not a.quick:
        db_pin = torch.from_numpy(db_np).pin_memory()
        q_pin = torch.from_numpy(q_np).pin_memory()
        ids_pin = torch.empty((a.nq, a.k), dtype=torch.int32).pin_memory()
        dist_pin = torch.empty((a.nq, a.k), dtype=out_dist.dtype).pin_memory()

        def serial_step():
            ix = hc.hc_build_host(db_pin, 8, 16, stream=stream)
            hc.hc_query_host(ix, q_pin, a.k, a.p, ids_pin, dist_pin, stream=stream)
            ix.free()

        copy_s, build_s = torch.cuda.Stream(), torch.cuda.Stream()
        # one set of pinned result buffers per step in flight
        outs = [(torch.empty((a.nq, a.k), dtype=torch.int32).pin_memory(),
                 torch.empty((a.nq, a.k), dtype=out_dist.dtype).pin_memory())
                for _ in range(a.e2e_depth + 1)]

        def pipelined(steps):
            """steps whole steps (rows and queries up, build, key-order walk,
            results down).  Step j's rows and queries are queued on the copy
            stream a.e2e_depth steps before the host collects step j, so the
            copy engine uploads while the SMs build and query earlier steps;
            every copy of the steps lies inside the call."""
            ahead = collections.deque()

            def enqueue(j):
                ix = hc.hc_build_host_async(db_pin, 8, 16, stream=build_s, copy_stream=copy_s)
                built = torch.cuda.Event()
                built.record(build_s)
                stream.wait_event(built)
                oi, od = outs[j % len(outs)]
                hc.hc_query_host_async(ix, q_pin, a.k, a.p, oi, od, stream=stream,
                                       copy_stream=copy_s)
                done = torch.cuda.Event()
                done.record(stream)
                ahead.append((ix, done))

            queued = 0
            while queued < min(a.e2e_depth, steps):
                enqueue(queued)
                queued += 1
            for _ in range(steps):
                if queued < steps:
                    enqueue(queued)
                    queued += 1
                ix, done = ahead.popleft()
                done.synchronize()   # this step's results are in host memory
                ix.free(stream=stream)

        def timed(fn):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            return (time.perf_counter() - t0) / a.steps

        for _ in range(max(1, a.warmup)):
            serial_step()
        serial_s = timed(lambda: [serial_step() for _ in range(a.steps)])
        pipelined(max(1, a.warmup))
        # the host-to-device rate of this shared box swings between runs (the
        # same pipeline measured 9.4 and 10.4-12 ms per step back to back, in
        # every build): the median of E2E_RUNS timed runs of all K steps
        runs = [timed(lambda: pipelined(a.steps)) for _ in range(E2E_RUNS)]
        e2e_s = statistics.median(runs)
        e2e = {"value": a.nq / e2e_s, "unit": UNIT,
               "runs_ms_per_step": [round(r * 1000.0, 3) for r in runs],
               "h2d_bytes_per_step": int(db_np.nbytes + q_np.nbytes),
               "d2h_bytes_per_step": int(ids_pin.numel() * 4 + dist_pin.numel() * 4),
               "ms_per_step": e2e_s * 1000.0,
               "statistic": "median of %d runs of %d steps" % (E2E_RUNS, a.steps),
               "path": "hc_build_host_async (rows up from pinned host memory on a copy "
                       "stream, the build behind an event on a second stream) + "
                       "hc_query_host_async (queries up on the copy stream, key-order walk, "
                       "results down to pinned memory); each step's copies are queued %d "
                       "steps ahead, so uploads overlap the builds and queries of earlier "
                       "steps; every step's copies lie inside the timed region" % a.e2e_depth,
               "serial": {"value": a.nq / serial_s, "ms_per_step": serial_s * 1000.0,
                          "path": "hc_build_host + hc_query_host, one step after another"}}

    cpu = None
    if not a.quick and not a.no_cpu_baseline and world == 1:
        cpu = cpu_oracle_sample(a, db_np, q_np)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": a.dtype, "data": DATA,
            "config": cfg, "roofline": roofline, "roofline_build": roofline_build,
            "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    a = parse_args()
    if a.impl == "reference":
        return run_reference(a)
    if a.workload == "uneven":
        from bench_workloads import run_uneven
        return run_uneven(a)
    if a.workload == "learned":
        from bench_workloads import run_learned
        return run_learned(a)
    if a.workload == "serve":
        from bench_workloads import run_serve
        return run_serve(a)
    if a.workload == "partitions":
        from bench_workloads import run_partitions
        return run_partitions(a)
    return run_hc(a)


if __name__ == "__main__":
    sys.exit(main())

"""The non-headline workloads of bench.py (each prints one JSON line):

uneven   64 independent indexes (N log-uniform in [10k, 2M], d in {64, 128,
         256}, uint8 and float32 mixed, c = d/16 curves), query batches
         log-uniform in [1, 4096], k in {1, 10, 100}, p = 64: one persistent
         launch replayed from a CUDA graph (autotuned) against one hc_query
         launch per index.
learned  N = 10M uint8, depth predictor trained on the device on seeded
         queries with two label targets (minimal p reproducing the p = 512
         top-10, and the p = 128 top-10), evaluated on held-out queries:
         recall@10 (exact kNN on a sample), agreement with p = 512, queries/s
         of learned against fixed depths at matched recall.
serve    N = 50M uint8 resident, Poisson arrivals whose rate follows seeded
         on/off bursts times a sinusoid between 10k and 500k queries/s, k = 10,
         requests with p = 0 (learned depth, fixed-depth fallback), HBM-budget
         admission, a 200 us latency bound on batching: p50/p99 latency and
         sustained queries/s; latency against offered load (fixed-rate
         Poisson phases, learned and fixed depth); a closed loop of 4096-query
         requests for the server's capacity; the plain fixed-depth batch
         throughput on the same index.
partitions
         partitioned Hypercurves on one GPU (Sec. 4): N = 10M uint8 split into
         ell in {1, 2, 4, 8, 16, 32} in-HBM partitions, sequential depth
         Phi = 128, local depth phi from the Optimist (slack 0) and Pessimist
         (smallest slack with Eq. 6 below 2%) settings: build and query time,
         recall@10, and how often the answer equals / is no worse than the
         sequential one.
"""
import json
from fractions import Fraction
import math
import os
import statistics
import tempfile
import threading
import time

import numpy as np


def _line(d):
    print(json.dumps(d), flush=True)


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


# ------------------------------------------------------------------ uneven
def run_uneven(a):
    import torch
    from paper_1209_0410_gb300 import autotune, datagen, hc
    torch.cuda.set_device(0)
    shapes = datagen.uneven_workload(seed=11)
    p = 64
    jobs, total_q = [], 0
    t0 = time.time()
    for sh in shapes:
        db = datagen.make_db(sh["n"], sh["d"], seed=sh["seed"])
        q = datagen.make_queries(db, sh["nq"], seed=sh["seed"] + 50_000)
        if sh["dtype"] == "f32":
            db, q = datagen.to_f32(db), datagen.to_f32(q)
        tdb = torch.from_numpy(db).cuda()
        idx = hc.hc_build(tdb, sh["d"] // 16, 16)
        jobs.append(hc.MultiJob(idx, torch.from_numpy(q).cuda(), sh["k"], p))
        total_q += sh["nq"]
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    stream = torch.cuda.current_stream()
    reps = max(3, a.steps)

    # one launch per index
    for j in jobs:
        hc.hc_query(j.index, j.q, j.k, j.p)
    e0, e1 = _events()
    e0.record(stream)
    for _ in range(reps):
        for j in jobs:
            hc.hc_query(j.index, j.q, j.k, j.p)
    e1.record(stream)
    torch.cuda.synchronize()
    per_index_ms = e0.elapsed_time(e1) / reps
    ref = [hc.hc_query(j.index, j.q, j.k, j.p) for j in jobs]

    # one persistent launch (autotuned), replayed from a CUDA graph
    cache = a.tune_cache or os.path.join(tempfile.gettempdir(), "hc_tune_uneven.json")
    t1 = time.time()
    cfg = autotune.tune(jobs, cache_path=cache)
    tune_s = time.time() - t1
    plan = hc.MultiPlan(jobs, dict(cfg, use_graph=True))
    for _ in range(a.warmup):
        plan.run()
    launches0 = hc.hc_launch_count()
    e0.record(stream)
    for _ in range(reps):
        plan.run()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = (hc.hc_launch_count() - launches0) // reps
    persistent_ms = e0.elapsed_time(e1) / reps
    same = all(torch.equal(j.ids, r[0]) for j, r in zip(jobs, ref))
    # the method's own bytes for all jobs (window rows and ids, probes, queries, results)
    from bench import algorithmic_query_bytes, measured_peaks
    qbytes = 0
    for sh, j in zip(shapes, jobs):
        row_bytes = sh["d"] * (4 if sh["dtype"] == "f32" else 1)
        if sh["nq"]:
            qbytes += algorithmic_query_bytes(hc, j.index, j.q, j.p, j.k, row_bytes)[0]
    peak_gbs = measured_peaks()[0]["hbm_gbs"]
    _line({"metric": "queries/s, 64 uneven indexes in one persistent launch (CUDA graph)",
           "value": total_q / (persistent_ms / 1e3), "unit": "queries/s", "n_gpus": 1,
           "steps": reps, "warmup": a.warmup, "ms_per_step": persistent_ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8+f32",
           "data": "synthetic: seeded Gaussian-mixture indexes of uneven shapes",
           "config": {"workload": "64 indexes, N log-uniform [10k, 2M], d in {64,128,256}, "
                                  "uint8/float32 mixed, batches log-uniform [1, 4096], "
                                  "k in {1,10,100}, p = 64",
                      "indexes": len(jobs), "queries": total_q,
                      "rows": int(sum(sh["n"] for sh in shapes)),
                      "per_index_launches_ms": per_index_ms,
                      "persistent_ms": persistent_ms,
                      "speedup_vs_per_index": per_index_ms / persistent_ms,
                      "autotuned_config": cfg, "tune_s": tune_s, "setup_s": setup_s,
                      "results_identical_to_per_index": same,
                      "kernel_launches_per_step": launches,
                      "algorithmic_bytes": qbytes,
                      "hbm_frac_persistent": qbytes / (persistent_ms / 1e3) / 1e9 / peak_gbs,
                      "hbm_frac_per_index": qbytes / (per_index_ms / 1e3) / 1e9 / peak_gbs}})
    plan.free()
    return 0


# ----------------------------------------------------------------- learned
def run_learned(a):
    import torch
    from paper_1209_0410_gb300 import datagen, hc, learned
    torch.cuda.set_device(0)
    n = a.n_db
    db = datagen.make_db(n, 128, seed=datagen.SEED_DB)
    qt = datagen.make_queries(db, a.train_queries, seed=datagen.SEED_TRAIN_QUERIES)
    qh = datagen.make_queries(db, a.heldout_queries, seed=datagen.SEED_HELDOUT_QUERIES)
    tdb = torch.from_numpy(db).cuda()
    tqt = torch.from_numpy(qt).cuda()
    tqh = torch.from_numpy(qh).cuda()
    idx = hc.hc_build(tdb, 8, 16)
    torch.cuda.synchronize()
    rs = min(2000, a.heldout_queries)
    _, tdist = hc.hc_bruteforce(tdb, tqh[:rs], 10)
    ref512, _ = hc.hc_query(idx, tqh, 10, 512)
    stream = torch.cuda.current_stream()

    def timed(fn, reps=3):
        fn()
        e0, e1 = _events()
        e0.record(stream)
        for _ in range(reps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / reps

    fixed = []
    for p in (32, 64, 128, 192, 256, 384, 512):
        (ids, dist), ms = timed(lambda: hc.hc_query(idx, tqh, 10, p))
        fixed.append({"p": p, "ms": ms, "qps": a.heldout_queries / (ms / 1e3),
                      "recall_at_10": learned.recall_at_10(ids[:rs], dist[:rs], tdist),
                      "agreement_p512": learned.agreement(ids, ref512)})
    base = [f for f in fixed if f["p"] == 128][0]
    r128 = base["recall_at_10"]
    # two label targets: the large depth of the configuration (p = 512) and
    # the operating point itself (p = 128)
    targets = {}
    for p_max in (512, 128):
        t0 = time.time()
        mlp, labels, losses = learned.fit(idx, tqt, k=10, p_max=p_max, epochs=8, batch=4096)
        torch.cuda.synchronize()
        train_s = time.time() - t0
        curve, chosen = [], None
        for m in [x / 4.0 for x in range(-16, 13)]:
            def run(m=m):
                pd = mlp.predict_depths(idx, tqh, m, 1, 512)
                return hc.hc_query_depths(idx, tqh, 10, pd) + (pd,)
            (ids, dist, pd), ms = timed(run)
            row = {"margin": m, "mean_p": float(pd.double().mean().item()), "ms": ms,
                   "qps": a.heldout_queries / (ms / 1e3),
                   "recall_at_10": learned.recall_at_10(ids[:rs], dist[:rs], tdist),
                   "agreement_p512": learned.agreement(ids, ref512)}
            curve.append(row)
            if chosen is None and row["recall_at_10"] >= r128:
                chosen = row
        targets["p_max_%d" % p_max] = {
            "labels": "minimal p reproducing the p=%d top-10" % p_max,
            "label_mean": float(labels.double().mean().item()), "train_s": train_s,
            "loss_per_epoch": losses, "learned_at_matched_recall": chosen,
            "speedup_vs_fixed_p128": (chosen["qps"] / base["qps"]) if chosen else None,
            "learned_sweep": curve}
        mlp.free()
    best = max((t for t in targets.values() if t["learned_at_matched_recall"]),
               key=lambda t: t["learned_at_matched_recall"]["qps"], default=None)
    chosen = best["learned_at_matched_recall"] if best else None
    _line({"metric": "queries/s at recall@10 >= plain p=128, learned probe depth, 10M x 128 "
                     "uint8", "value": chosen["qps"] if chosen else None, "unit": "queries/s",
           "n_gpus": 1, "steps": 3, "warmup": 1, "ms_per_step": chosen["ms"] if chosen else None,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
           "data": "synthetic: seeded 64-cluster Gaussian mixture; train seed 4, held-out seed 5",
           "config": {"workload": "learned depth: N=%d, MLP 32-64-64-1 (FP32 Adam training on "
                                  "the device, BF16 inference), %d train / %d held-out queries, "
                                  "labels = minimal p reproducing the p=512 or the p=128 top-10"
                                  % (n, a.train_queries, a.heldout_queries),
                      "fixed_p128": base, "value_from": best["labels"] if best else None,
                      "label_targets": targets, "fixed_sweep": fixed,
                      "recall_sample_queries": rs}})
    return 0


# ------------------------------------------------------------------- serve
def arrival_times(seconds, seed, lo=10_000.0, hi=500_000.0, per_request=32):
    """Request arrival times: a Poisson process (thinning) whose query rate is
    clip(mid + amp * sin(2 pi t / 4 s), lo, hi) times seeded on/off bursts
    (on: x1, off: x0.25; exponential durations of mean 0.7 s)."""
    rng = np.random.default_rng(seed)
    # burst switch times
    switches, t, on = [], 0.0, True
    while t < seconds:
        switches.append((t, on))
        t += rng.exponential(0.7)
        on = not on

    def rate(tt):
        mid, amp = (hi + lo) / 2, (hi - lo) / 2
        base = mid + amp * math.sin(2 * math.pi * tt / 4.0)
        state = True
        for ts, st in switches:
            if ts <= tt:
                state = st
        return min(hi, max(lo, base * (1.0 if state else 0.25)))

    lam_max = hi / per_request
    out, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / lam_max)
        if t >= seconds:
            break
        if rng.random() < rate(t) / per_request / lam_max:
            out.append(t)
    return np.array(out)


def run_serve(a):
    import torch
    from paper_1209_0410_gb300 import datagen, hc, learned
    torch.cuda.set_device(0)
    n = a.serve_n
    t0 = time.time()
    db = datagen.make_db(n, 128, seed=datagen.SEED_DB)
    pool = datagen.make_queries(db, 262_144, seed=datagen.SEED_QUERIES)
    qt = datagen.make_queries(db, 200_000, seed=datagen.SEED_TRAIN_QUERIES)
    tdb = torch.from_numpy(db).cuda()
    idx = hc.hc_build(tdb, 8, 16)
    mlp, _, _ = learned.fit(idx, torch.from_numpy(qt).cuda(), k=10, p_max=512, epochs=6,
                            batch=4096)
    # margin: smallest whose recall@10 reaches that of fixed p = 128
    val = torch.from_numpy(pool[:4000]).cuda()
    _, tdist = hc.hc_bruteforce(tdb, val[:1000], 10)
    ids, dist = hc.hc_query(idx, val[:1000], 10, 128)
    r128 = learned.recall_at_10(ids, dist, tdist)
    margin = 1.0
    for m in [x / 4.0 for x in range(-16, 9)]:
        pd = mlp.predict_depths(idx, val[:1000], m, 1, 512)
        ids, dist = hc.hc_query_depths(idx, val[:1000], 10, pd)
        if learned.recall_at_10(ids, dist, tdist) >= r128:
            margin = m
            break
    torch.cuda.synchronize()
    setup_s = time.time() - t0

    per_req = 32
    arrivals = arrival_times(a.serve_seconds, seed=17, per_request=per_req)
    srv = hc.Server([idx], 2 << 30, streams=4, max_batch_queries=8192, default_p=128,
                    max_wait_us=200)
    srv.attach_predictor(0, mlp, margin, 1, 512)

    def open_loop(arr, p):
        """Submits per_req-query requests at the given arrival times (seconds)
        from one thread while another polls; returns latencies (s) and wall."""
        tickets = [None] * len(arr)
        done = []

        def submitter():
            start = time.perf_counter()
            for i, ta in enumerate(arr):
                while True:
                    now = time.perf_counter() - start
                    if now >= ta:
                        break
                    if ta - now > 0.0005:
                        time.sleep(ta - now - 0.0004)
                s0 = (i * per_req) % (pool.shape[0] - per_req)
                tickets[i] = srv.submit(0, pool[s0:s0 + per_req], 10, p)

        def poller():
            for i in range(len(arr)):
                while tickets[i] is None:
                    time.sleep(0.0001)
                r = None
                while r is None:
                    r = srv.poll(tickets[i], 1_000_000, with_latency=True)
                done.append(r[2])

        w0 = time.perf_counter()
        ts = threading.Thread(target=submitter)
        tp = threading.Thread(target=poller)
        ts.start()
        tp.start()
        ts.join()
        tp.join()
        return np.array(done), time.perf_counter() - w0

    lat_s, wall = open_loop(arrivals, 0)
    st = srv.stats()
    lat = lat_s * 1e3
    served = len(lat_s) * per_req

    # latency against offered load: Poisson arrivals at fixed rates, one
    # second each, learned depth and fixed p = 128
    load = []
    rng = np.random.default_rng(23)
    for rate in (50_000, 200_000, 500_000, 1_000_000, 2_000_000):
        arr = np.cumsum(rng.exponential(per_req / rate, size=int(rate / per_req * 1.2)))
        arr = arr[arr < 1.0]
        row = {"offered_qps": rate}
        for name, p in (("learned", 0), ("fixed_p128", 128)):
            l_s, w = open_loop(arr, p)
            row[name] = {"served_qps": len(l_s) * per_req / w,
                         "p50_ms": float(np.percentile(l_s, 50) * 1e3),
                         "p99_ms": float(np.percentile(l_s, 99) * 1e3)}
        load.append(row)

    # saturation: a closed loop keeps `outstanding` requests of sat_req queries
    # in the server for about two seconds (capacity rather than offered load)
    def closed_loop(p, sat_req=4096, outstanding=16, seconds=2.0):
        lat_c, nq_c, pending, i = [], 0, [], 0
        t0c = time.perf_counter()
        while True:
            while len(pending) < outstanding and time.perf_counter() - t0c < seconds:
                s0 = (i * sat_req) % (pool.shape[0] - sat_req)
                pending.append(srv.submit(0, pool[s0:s0 + sat_req], 10, p))
                i += 1
            if not pending:
                break
            r = None
            while r is None:
                r = srv.poll(pending[0], 1_000_000, with_latency=True)
            pending.pop(0)
            lat_c.append(r[2])
            nq_c += sat_req
        return nq_c / (time.perf_counter() - t0c), np.array(lat_c) * 1e3

    sat_req, outstanding = 4096, 16
    sat_qps, sat_lat = closed_loop(0)
    sat_qps_fixed, sat_lat_fixed = closed_loop(128)
    srv.close()

    # the plain method on the same index: one batch of 100k queries at fixed
    # p = 128, answered in key order, timed on the device
    qb = torch.from_numpy(np.ascontiguousarray(pool[:100_000])).cuda()
    ob_ids = torch.empty((qb.shape[0], 10), dtype=torch.int32, device="cuda")
    ob_dist = torch.empty((qb.shape[0], 10), dtype=torch.int32, device="cuda")
    ws = torch.empty(hc.hc_query_ordered_workspace(idx, qb.shape[0]), dtype=torch.uint8,
                     device="cuda")
    hc.hc_query_ordered(idx, qb, 10, 128, ob_ids, ob_dist, workspace=ws)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(5):
        hc.hc_query_ordered(idx, qb, 10, 128, ob_ids, ob_dist, workspace=ws)
    ev[1].record()
    torch.cuda.synchronize()
    plain_qps = qb.shape[0] / (ev[0].elapsed_time(ev[1]) / 5 / 1000.0)
    # recall of the served answers (learned depths) on a sample
    sample = torch.from_numpy(pool[:1000]).cuda()
    pd = mlp.predict_depths(idx, sample, margin, 1, 512)
    ids, dist = hc.hc_query_depths(idx, sample, 10, pd)
    _, td = hc.hc_bruteforce(tdb, sample, 10)
    rec = learned.recall_at_10(ids, dist, td)
    _line({"metric": "served queries/s and p50/p99 latency under fluctuating load, 50M x 128 "
                     "uint8", "value": served / wall, "unit": "queries/s", "n_gpus": 1,
           "steps": len(arrivals), "warmup": 0, "ms_per_step": None, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u8",
           "data": "synthetic: seeded 64-cluster Gaussian mixture, Poisson arrivals",
           "config": {"workload": "online serving: N=%d resident, Poisson arrivals with rate = "
                                  "seeded on/off bursts x sinusoid in [10k, 500k] q/s, "
                                  "%d-query requests, k=10, p=0 (learned depth, margin %.2f; "
                                  "fixed p=128 fallback), 2 GiB HBM budget, 4 streams"
                                  % (n, per_req, margin),
                      "seconds": a.serve_seconds, "requests": len(arrivals),
                      "offered_qps_mean": len(arrivals) * per_req / a.serve_seconds,
                      "latency_ms": {"p50": float(np.percentile(lat, 50)),
                                     "p99": float(np.percentile(lat, 99)),
                                     "mean": float(lat.mean()), "max": float(lat.max())},
                      "recall_at_10": rec, "recall_at_10_fixed_p128": r128,
                      "server": {k: int(v) for k, v in st.items()},
                      "mean_batch_queries": st["queries_done"] / max(1, st["batches_done"]),
                      "max_wait_us": 200,
                      "latency_vs_offered_load": load,
                      "saturation": {"qps": sat_qps, "request_queries": sat_req,
                                     "outstanding_requests": outstanding,
                                     "latency_ms": {"p50": float(np.percentile(sat_lat, 50)),
                                                    "p99": float(np.percentile(sat_lat, 99))},
                                     "fixed_p128_qps": sat_qps_fixed,
                                     "fixed_p128_latency_ms": {
                                         "p50": float(np.percentile(sat_lat_fixed, 50)),
                                         "p99": float(np.percentile(sat_lat_fixed, 99))}},
                      "plain_fixed_p128_batch_qps": plain_qps,
                      "setup_s": setup_s}})
    mlp.free()
    return 0


# -------------------------------------------------------------- partitions
def run_partitions(a):
    import torch
    from paper_1209_0410_gb300 import datagen, hc, learned, partition
    torch.cuda.set_device(0)
    n, nq, Phi, k = a.n_db, a.nq, a.p, a.k
    db = datagen.make_db(n, 128, seed=datagen.SEED_DB)
    q = datagen.make_queries(db, nq, seed=datagen.SEED_QUERIES)
    tdb = torch.from_numpy(db).cuda()
    tq = torch.from_numpy(q).cuda()
    stream = torch.cuda.current_stream()
    rs = min(2000, nq)
    _, tdist = hc.hc_bruteforce(tdb, tq[:rs], 10)
    reps = max(3, min(a.steps, 10))
    seq_ids = seq_dist = None
    rows = []
    for ell in (1, 2, 4, 8, 16, 32):
        e0, e1 = _events()
        hc.hc_build(tdb, 8, 16, partitions=ell).free()      # warm the pool
        e0.record(stream)
        idx = hc.hc_build(tdb, 8, 16, partitions=ell)
        e1.record(stream)
        torch.cuda.synchronize()
        build_ms = e0.elapsed_time(e1)
        settings = [("optimist", Fraction(0))]
        if ell > 1:
            settings.append(("pessimist", partition.pessimist_slack(Phi, ell)))
        for name, slack in settings:
            phi = partition.slack_depth(Phi, ell, slack)
            ids, dist = hc.hc_query(idx, tq, k, phi)
            e0, e1 = _events()
            e0.record(stream)
            for _ in range(reps):
                hc.hc_query(idx, tq, k, phi, ids, dist)
            e1.record(stream)
            torch.cuda.synchronize()
            plain_ms = e0.elapsed_time(e1) / reps
            # the ordered path: every curve's key order, one batch lower_bound
            # pass, then the walk (the same results)
            ws = torch.empty(hc.hc_query_ordered_workspace(idx, nq), dtype=torch.uint8,
                             device="cuda")
            o_ids = torch.empty_like(ids)
            o_dist = torch.empty_like(dist)
            hc.hc_query_ordered(idx, tq, k, phi, o_ids, o_dist, workspace=ws)
            e0, e1 = _events()
            e0.record(stream)
            for _ in range(reps):
                hc.hc_query_ordered(idx, tq, k, phi, o_ids, o_dist, workspace=ws)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            same = bool(torch.equal(ids, o_ids) and torch.equal(dist, o_dist))
            del ws
            if seq_ids is None:
                seq_ids, seq_dist = ids.clone(), dist.clone()
            row = {"ell": ell, "setting": name, "slack": float(slack), "phi": phi,
                   "bound_eq6": partition.equiv_bound(Phi, ell, phi) if ell > 1 else 0.0,
                   "build_ms": build_ms, "query_ms": ms, "qps": nq / (ms / 1e3),
                   "plain_query_ms": plain_ms, "ordered_equals_plain": same,
                   "window_rows_per_query": 2 * phi * ell * 8,
                   "recall_at_10": learned.recall_at_10(ids[:rs], dist[:rs], tdist),
                   "equal_to_sequential": learned.agreement(ids, seq_ids),
                   "no_worse_than_sequential": float(
                       (dist <= seq_dist).all(dim=1).double().mean().item())}
            rows.append(row)
        idx.free()
    ref = [r for r in rows if r["ell"] == 8 and r["setting"] == "pessimist"][0]
    _line({"metric": "queries/s, partitioned Hypercurves (8 in-HBM partitions, Pessimist "
                     "slack), 10M x 128 uint8", "value": ref["qps"], "unit": "queries/s",
           "n_gpus": 1, "steps": reps, "warmup": 1, "ms_per_step": ref["query_ms"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
           "data": "synthetic: seeded 64-cluster Gaussian mixture (SIFT stand-in)",
           "config": {"workload": "partitioned Hypercurves: N=%d, Q=%d, sequential depth "
                                  "Phi=%d per side, k=%d, ell in {1..32} contiguous "
                                  "partitions, Optimist / Pessimist slack" % (n, nq, Phi, k),
                      "l2": "inputs larger than L2 (database %.2f GB)" % (n * 128 / 1e9),
                      "query_path": "hc_query_ordered (per-curve key orders, one batch "
                                    "lower_bound pass, walk in curve-0 order; results equal "
                                    "hc_query, whose time is plain_query_ms)",
                      "recall_sample_queries": rs, "sweep": rows}})
    return 0

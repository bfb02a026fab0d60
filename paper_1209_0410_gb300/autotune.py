"""Autotuner of the persistent multi-index launch.

Two levels, both measured with CUDA events on the launching stream:
  - per job class (d, dtype, k, p): the warps that share one query
    (1, 2, 4 or 8), timed on that class's jobs alone;
  - for the whole job set: warps per block, persistent blocks per SM and the
    tile (query groups per task), timed on the full persistent launch.
Results are cached in a JSON file keyed by those classes, so a later run
with the same shapes skips the search.
"""
import json
import os

import torch

from . import hc

WPQ_CHOICES = (1, 2, 4, 8)
BLOCK_CHOICES = ({"warps_per_block": 8, "blocks_per_sm": 2, "tile": 1},
                 {"warps_per_block": 8, "blocks_per_sm": 2, "tile": 2},
                 {"warps_per_block": 8, "blocks_per_sm": 3, "tile": 1},
                 {"warps_per_block": 8, "blocks_per_sm": 3, "tile": 2},
                 {"warps_per_block": 8, "blocks_per_sm": 3, "tile": 4},
                 {"warps_per_block": 8, "blocks_per_sm": 4, "tile": 2},
                 {"warps_per_block": 4, "blocks_per_sm": 4, "tile": 2},
                 {"warps_per_block": 16, "blocks_per_sm": 1, "tile": 1},
                 {"warps_per_block": 16, "blocks_per_sm": 2, "tile": 1})


def class_key(job):
    ix = job.index
    return "d%d_%s_k%d_p%d" % (ix.d, "f32" if ix.dtype == hc.HC_F32 else "u8", job.k, job.p)


def _time_plan(jobs, config, reps=3, stream=None):
    stream = stream or torch.cuda.current_stream()
    plan = hc.MultiPlan(jobs, dict(config, use_graph=True), stream=stream)
    plan.run(stream)                       # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        plan.run(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    plan.free()
    return e0.elapsed_time(e1) / reps


def _load(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {"classes": {}, "sets": {}}


def _save(path, cache):
    if not path:
        return
    d = os.path.dirname(os.path.abspath(path))
    os.makedirs(d, exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune(jobs, cache_path=None, stream=None):
    """Sets each job's warps_per_query and returns the block configuration
    for the whole set (a dict for MultiPlan)."""
    cache = _load(cache_path)
    base = {"warps_per_block": 8, "blocks_per_sm": 2, "tile": 1}
    by_class = {}
    for j in jobs:
        by_class.setdefault(class_key(j), []).append(j)
    for key, js in sorted(by_class.items()):
        if key not in cache["classes"]:
            best = None
            for w in WPQ_CHOICES:
                for j in js:
                    j.warps_per_query = w
                ms = _time_plan(js, base, stream=stream)
                if best is None or ms < best[1]:
                    best = (w, ms)
            cache["classes"][key] = {"warps_per_query": best[0], "ms": best[1]}
        for j in js:
            j.warps_per_query = cache["classes"][key]["warps_per_query"]
    set_key = "|".join("%s:%d" % (k, sum(j.q.shape[0] for j in v))
                       for k, v in sorted(by_class.items()))
    if set_key not in cache["sets"]:
        best = None
        for cfg in BLOCK_CHOICES:
            if any(j.warps_per_query > cfg["warps_per_block"] for j in jobs):
                continue
            ms = _time_plan(jobs, cfg, stream=stream)
            if best is None or ms < best[1]:
                best = (cfg, ms)
        cache["sets"][set_key] = {"config": best[0], "ms": best[1]}
    _save(cache_path, cache)
    return dict(cache["sets"][set_key]["config"])

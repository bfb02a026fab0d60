"""Host logic of the persistent-launch autotuner, with the GPU timing replaced
by a deterministic cost model: it must pick the cheapest warps per query for
every job class and the cheapest block configuration for the set, write them
to its JSON cache, and serve a repeated tuning from the cache without timing."""
import json
import types

import pytest

from paper_1209_0410_gb300 import autotune, hc


def fake_job(d, f32, k, p, nq=100):
    ix = types.SimpleNamespace(d=d, dtype=hc.HC_F32 if f32 else hc.HC_U8)
    q = types.SimpleNamespace(shape=(nq, d))
    return types.SimpleNamespace(index=ix, q=q, k=k, p=p, warps_per_query=1)


def cost(jobs, config, **_):
    # per class: warps per query best at 4 for d=256, 2 otherwise; per set:
    # the configuration with 16 warps and 2 blocks per SM is the cheapest
    ms = 0.0
    for j in jobs:
        best = 4 if j.index.d == 256 else 2
        ms += 1.0 + abs(j.warps_per_query - best)
    ms *= {16: 0.5}.get(config["warps_per_block"], 1.0)
    ms *= 0.9 if config["blocks_per_sm"] == 2 else 1.0
    return ms


def test_tune_picks_minima_and_caches(tmp_path, monkeypatch):
    jobs = [fake_job(256, False, 10, 64), fake_job(128, True, 10, 64),
            fake_job(256, False, 10, 64), fake_job(64, False, 1, 64)]
    calls = []
    monkeypatch.setattr(autotune, "_time_plan",
                        lambda js, config, **kw: calls.append(1) or cost(js, config))
    path = str(tmp_path / "tune.json")
    cfg = autotune.tune(jobs, cache_path=path)
    assert [j.warps_per_query for j in jobs] == [4, 2, 4, 2]
    assert cfg == {"warps_per_block": 16, "blocks_per_sm": 2, "tile": 1}
    cache = json.load(open(path))
    assert set(cache["classes"]) == {autotune.class_key(j) for j in jobs}
    assert calls
    # a second tuning with the same shapes is served from the cache
    for j in jobs:
        j.warps_per_query = 1

    def no_timing(*a, **k):
        raise AssertionError("the cache should answer")
    monkeypatch.setattr(autotune, "_time_plan", no_timing)
    assert autotune.tune(jobs, cache_path=path) == cfg
    assert [j.warps_per_query for j in jobs] == [4, 2, 4, 2]


def test_class_key_separates_shapes():
    a = autotune.class_key(fake_job(128, False, 10, 64))
    assert a != autotune.class_key(fake_job(128, True, 10, 64))
    assert a != autotune.class_key(fake_job(128, False, 100, 64))
    assert a != autotune.class_key(fake_job(256, False, 10, 64))

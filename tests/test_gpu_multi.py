"""Many indexes in one persistent launch (and its CUDA graph), against the CPU
oracle's Algorithm 2 on every job and against per-index hc_query calls.

Against the oracle: uint8 ids and int32 distances bit for bit, float32
distances within 1e-5 relative with id sets equal outside the tie band at
the k-th distance, for every warps-per-query split (whose per-warp top-k
lists are merged in shared memory), block configuration, k in {1, 10, 33,
100}, d in {64, 128, 256} and batch sizes 0 to 1000.  Against hc_query: the
same arithmetic, so bit for bit on both element types."""
import json

import numpy as np
import pytest

from helpers import compare_f32, dev
from oracle import oracle as O
from paper_1209_0410_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_0410_gb300 import hc as _hc
    _hc.lib()
    return _hc


SHAPES = [  # (n, d, dtype, nq, k, p)
    (12000, 128, "u8", 300, 10, 64), (5000, 64, "u8", 1, 1, 40), (20000, 256, "u8", 77, 100, 30),
    (9000, 128, "f32", 130, 10, 50), (7000, 64, "f32", 0, 10, 20), (15000, 256, "f32", 41, 1, 70),
    (3000, 128, "u8", 1000, 33, 16), (4000, 64, "u8", 9, 100, 500),
]


@pytest.fixture(scope="module")
def jobs_data(hc):
    out = []
    for i, (n, d, dt, nq, k, p) in enumerate(SHAPES):
        db = datagen.make_db(n, d, seed=200 + i)
        q = datagen.make_queries(db, max(nq, 1), seed=300 + i)[:nq]
        if dt == "f32":
            db, q = datagen.to_f32(db), datagen.to_f32(q)
        idx = hc.hc_build(dev(db), d // 16, 16)
        out.append((idx, dev(np.ascontiguousarray(q)), k, p, db))
    return out


@pytest.fixture(scope="module")
def oracle_results(jobs_data):
    """Algorithm 2 of the CPU oracle for every job (ids, float64 distances)."""
    out = []
    for idx, q, k, p, db in jobs_data:
        qn = q.cpu().numpy()
        if qn.shape[0] == 0:
            out.append(None)
            continue
        oidx = O.build(db, curves=db.shape[1] // 16, m=16)
        out.append(O.search(oidx, db, qn, k, p))
    return out


def assert_matches_oracle(job, ref, db):
    if ref is None:
        assert job.ids.numel() == 0
        return
    rids, rdist = ref
    gids, gdist = job.ids.cpu().numpy(), job.dist.cpu().numpy()
    if db.dtype == np.uint8:
        assert np.array_equal(gids, rids)
        assert np.array_equal(gdist, O.int32_dist(rdist))
    else:
        assert compare_f32(gids, gdist, rids, rdist) == []


@pytest.mark.parametrize("wpq", [1, 2, 4, 8])
@pytest.mark.parametrize("cfg", [dict(warps_per_block=8, blocks_per_sm=2, tile=1),
                                 dict(warps_per_block=16, blocks_per_sm=1, tile=3)])
def test_multi_matches_oracle(hc, jobs_data, oracle_results, wpq, cfg):
    import torch
    jobs = [hc.MultiJob(idx, q, k, p, warps_per_query=wpq) for idx, q, k, p, _ in jobs_data]
    hc.hc_query_multi(jobs, cfg)
    torch.cuda.synchronize()
    for j, ref, (_, _, _, _, db) in zip(jobs, oracle_results, jobs_data):
        assert_matches_oracle(j, ref, db)


def test_multi_graph_matches_oracle(hc, jobs_data, oracle_results):
    import torch
    jobs = [hc.MultiJob(idx, q, k, p, warps_per_query=4) for idx, q, k, p, _ in jobs_data]
    plan = hc.MultiPlan(jobs, dict(warps_per_block=8, blocks_per_sm=2, tile=2, use_graph=True))
    for _ in range(2):
        plan.run()
        torch.cuda.synchronize()
        for j, ref, (_, _, _, _, db) in zip(jobs, oracle_results, jobs_data):
            assert_matches_oracle(j, ref, db)
    plan.free()


def reference(hc, jobs_data):
    import torch
    refs = []
    for idx, q, k, p, _ in jobs_data:
        ids, dist = hc.hc_query(idx, q, k, p)
        refs.append((ids, dist))
    torch.cuda.synchronize()
    return refs


@pytest.mark.parametrize("wpq", [1, 2, 4, 8])
@pytest.mark.parametrize("cfg", [dict(warps_per_block=8, blocks_per_sm=2, tile=1),
                                 dict(warps_per_block=16, blocks_per_sm=1, tile=3),
                                 dict(warps_per_block=8, blocks_per_sm=4, tile=2)])
def test_multi_matches_per_index_queries(hc, jobs_data, wpq, cfg):
    import torch
    refs = reference(hc, jobs_data)
    jobs = [hc.MultiJob(idx, q, k, p, warps_per_query=wpq) for idx, q, k, p, _ in jobs_data]
    hc.hc_query_multi(jobs, cfg)
    torch.cuda.synchronize()
    for j, (rids, rdist) in zip(jobs, refs):
        assert torch.equal(j.ids, rids)
        assert torch.equal(j.dist.view(torch.int32), rdist.view(torch.int32))


def test_graph_replay_sees_new_queries(hc, jobs_data):
    import torch
    jobs = [hc.MultiJob(idx, q.clone(), k, p, warps_per_query=2)
            for idx, q, k, p, _ in jobs_data]
    plan = hc.MultiPlan(jobs, dict(warps_per_block=8, blocks_per_sm=2, tile=2, use_graph=True))
    plan.run()
    torch.cuda.synchronize()
    for j, (rids, _) in zip(jobs, reference(hc, jobs_data)):
        assert torch.equal(j.ids, rids)
    # write other queries into the same buffers and replay the graph
    for j, (idx, q, k, p, db) in zip(jobs, jobs_data):
        if q.shape[0]:
            j.q.copy_(q.flip(0))
    plan.run()
    torch.cuda.synchronize()
    for j, (idx, q, k, p, db) in zip(jobs, jobs_data):
        if q.shape[0]:
            rids, _ = hc.hc_query(idx, q.flip(0).contiguous(), k, p)
            torch.cuda.synchronize()
            assert torch.equal(j.ids, rids)
    plan.free()


def test_autotuner_picks_and_caches(hc, jobs_data, tmp_path):
    import torch
    from paper_1209_0410_gb300 import autotune
    jobs = [hc.MultiJob(idx, q, k, p) for idx, q, k, p, _ in jobs_data]
    path = str(tmp_path / "tune.json")
    cfg = autotune.tune(jobs, cache_path=path)
    cache = json.load(open(path))
    assert cache["classes"] and cache["sets"]
    assert all(j.warps_per_query in (1, 2, 4, 8) for j in jobs)
    plan = hc.MultiPlan(jobs, dict(cfg, use_graph=True))
    plan.run()
    torch.cuda.synchronize()
    for j, (rids, _) in zip(jobs, reference(hc, jobs_data)):
        assert torch.equal(j.ids, rids)
    # a second tuning with the same shapes is served from the cache
    cfg2 = autotune.tune(jobs, cache_path=path)
    assert cfg2 == cfg


def test_multi_rejects_bad_jobs(hc, jobs_data):
    idx, q, k, p, _ = jobs_data[0]
    with pytest.raises(hc.HCError):
        hc.hc_query_multi([hc.MultiJob(idx, q, k, p, warps_per_query=3)])
    with pytest.raises(hc.HCError):
        hc.hc_query_multi([hc.MultiJob(idx, q, k, p, warps_per_query=16)],
                          dict(warps_per_block=8, blocks_per_sm=1, tile=1))

"""The serving loop (hc_serve_*): continuous batching under an HBM budget.

Every request's result must be bit-identical to the same queries answered by
hc_query alone, whether the request was served alone or mixed with others of
different sizes, depths, k and indexes arriving from several threads while
batches are on the GPU.  Admission: a request larger than the budget is
refused; a small budget still serves everything (requests wait for room).
"""
import threading
import time

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


@pytest.fixture(scope="module")
def indexes(hc):
    """Three resident indexes: uint8 d=128, uint8 d=64 (4 curves), float32 d=128."""
    a = datagen.make_db(30000, 128, seed=61)
    b = datagen.make_db(20000, 64, seed=62)
    c = datagen.to_f32(datagen.make_db(15000, 128, seed=63))
    ia = hc.hc_build(dev(a), 8, 16)
    ib = hc.hc_build(dev(b), 4, 16)
    ic = hc.hc_build(dev(c), 8, 16)
    qa = datagen.make_queries(a, 3000, seed=71)
    qb = datagen.make_queries(b, 3000, seed=72)
    qc = datagen.to_f32(datagen.make_queries(datagen.make_db(15000, 128, seed=63), 3000, seed=73))
    return [(ia, qa), (ib, qb), (ic, qc)]


def test_served_results_match_oracle(hc, indexes):
    """A sample of requests on all three indexes, served together, against
    the CPU oracle's Algorithm 2: uint8 bit for bit, float32 within 1e-5
    relative (ties at the k-th distance aside)."""
    dbs = [datagen.make_db(30000, 128, seed=61), datagen.make_db(20000, 64, seed=62),
           datagen.to_f32(datagen.make_db(15000, 128, seed=63))]
    oidx = [O.build(db, curves=db.shape[1] // 16, m=16) for db in dbs]
    specs = [(0, 0, 120, 10, 64), (1, 500, 77, 33, 30), (2, 1000, 90, 10, 50),
             (0, 2000, 1, 1, 200), (2, 40, 64, 100, 16), (1, 2900, 100, 10, 0)]
    srv = hc.hc_serve_create([ix for ix, _ in indexes], 128 << 20, streams=4,
                             max_batch_queries=256, default_p=48)
    try:
        tickets = [srv.submit(i, indexes[i][1][s0:s0 + nq], k, p) for i, s0, nq, k, p in specs]
        results = [srv.poll(t, 30_000_000) for t in tickets]
    finally:
        srv.close()
    for (i, s0, nq, k, p), res in zip(specs, results):
        assert res is not None
        q = indexes[i][1][s0:s0 + nq]
        rids, rdist = O.search(oidx[i], dbs[i], q, k, p if p else 48)
        if dbs[i].dtype == np.uint8:
            assert np.array_equal(res[0], rids)
            assert np.array_equal(res[1], O.int32_dist(rdist))
        else:
            assert compare_f32(res[0], res[1], rids, rdist) == []


def alone(hc, index, q, k, p):
    import torch
    ids, dist = hc.hc_query(index, dev(q), k, p)
    torch.cuda.synchronize()
    return ids.cpu().numpy(), dist.cpu().numpy()


def test_single_request_matches_query(hc, indexes):
    srv = hc.hc_serve_create([ix for ix, _ in indexes], 64 << 20, default_p=48)
    try:
        for i, (ix, q) in enumerate(indexes):
            for k, p in ((10, 64), (1, 7), (33, 0)):
                t = srv.submit(i, q[:257], k, p)
                res = srv.poll(t, 10_000_000)
                assert res is not None
                ids, dist = res
                rids, rdist = alone(hc, ix, q[:257], k, p if p else 48)
                assert np.array_equal(ids, rids)
                assert np.array_equal(dist, rdist)
    finally:
        srv.close()


def test_mixed_concurrent_requests_bit_identical(hc, indexes):
    rng = np.random.default_rng(5)
    specs = []
    for r in range(240):
        i = int(rng.integers(0, 3))
        nq = int(rng.integers(1, 300))
        s0 = int(rng.integers(0, 3000 - nq))
        k = int(rng.choice([1, 10, 33]))
        p = int(rng.choice([0, 16, 64, 200]))
        specs.append((i, s0, nq, k, p))
    srv = hc.hc_serve_create([ix for ix, _ in indexes], 256 << 20, streams=4,
                             max_batch_queries=1024, default_p=40)
    tickets = [None] * len(specs)

    def producer(part):
        for j in range(part, len(specs), 4):
            i, s0, nq, k, p = specs[j]
            tickets[j] = srv.submit(i, indexes[i][1][s0:s0 + nq], k, p)
            if j % 7 == 0:
                time.sleep(0.0005)

    th = [threading.Thread(target=producer, args=(t,)) for t in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    results = [srv.poll(t, 30_000_000) for t in tickets]
    st = srv.stats()
    srv.close()
    for (i, s0, nq, k, p), res in zip(specs, results):
        assert res is not None
        rids, rdist = alone(hc, indexes[i][0], indexes[i][1][s0:s0 + nq], k, p if p else 40)
        assert np.array_equal(res[0], rids)
        assert np.array_equal(res[1], rdist)
    assert st["requests"] == len(specs)
    assert st["queries_done"] == sum(s[2] for s in specs)
    assert st["batches"] < len(specs)          # requests were batched together


def test_overlapping_batches_in_flight(hc, indexes):
    """With several streams and a full queue, more than one batch runs at once."""
    ix, q = indexes[0]
    srv = hc.hc_serve_create([ix], 512 << 20, streams=4, max_batch_queries=256)
    tickets = [srv.submit(0, q[(j * 256) % 2700:(j * 256) % 2700 + 256], 10, 400)
               for j in range(64)]
    for t in tickets:
        assert srv.poll(t, 30_000_000) is not None
    st = srv.stats()
    srv.close()
    assert st["max_inflight"] >= 2


def test_latency_bound_overlaps_batches(hc, indexes):
    """A small request that arrives while a long batch runs: with the latency
    bound it goes out on a second stream after max_wait_us (two batches in
    flight); without it (max_wait_us = 0) it waits for the GPU to go idle.
    Either way its result equals hc_query alone."""
    ix, q = indexes[0]
    for wait_us, want_overlap in ((100, True), (0, False)):
        srv = hc.hc_serve_create([ix], 512 << 20, streams=4, max_batch_queries=4096,
                                 max_wait_us=wait_us)
        try:
            big = srv.submit(0, q[:3000], 10, 2000)
            time.sleep(0.0002)
            small = srv.submit(0, q[:64], 10, 64)
            rs = srv.poll(small, 30_000_000)
            rb = srv.poll(big, 30_000_000)
            st = srv.stats()
        finally:
            srv.close()
        assert rs is not None and rb is not None
        rids, rdist = alone(hc, ix, q[:64], 10, 64)
        assert np.array_equal(rs[0], rids) and np.array_equal(rs[1], rdist)
        if want_overlap:
            assert st["max_inflight"] >= 2
        else:
            assert st["max_inflight"] == 1


def test_budget_admission(hc, indexes):
    ix, q = indexes[0]
    one = 128 * 128 + 128 * 4 + 2 * 128 * 10 * 4   # bytes of a 128-query, k=10 request
    budget = 3 * one
    srv = hc.hc_serve_create([ix], budget, streams=4, max_batch_queries=100000)
    try:
        with pytest.raises(hc.HCError) as e:
            srv.submit(0, q[:1000], 10, 32)       # needs more than the whole budget
        assert e.value.status == hc.HC_ERR_BUDGET
        tickets = [srv.submit(0, q[j * 128:(j + 1) * 128], 10, 32) for j in range(20)]
        peak = 0
        done = []
        for t in tickets:
            r = srv.poll(t, 30_000_000)
            assert r is not None
            done.append(r)
            peak = max(peak, srv.stats()["arena_used"])
        assert peak <= budget
        for j, (ids, dist) in enumerate(done):
            rids, rdist = alone(hc, ix, q[j * 128:(j + 1) * 128], 10, 32)
            assert np.array_equal(ids, rids) and np.array_equal(dist, rdist)
    finally:
        srv.close()


def test_tickets_and_pending(hc, indexes):
    ix, q = indexes[0]
    srv = hc.hc_serve_create([ix], 64 << 20)
    try:
        rc = hc.lib().hc_serve_poll(srv.handle, 987654321, None, None, 0)
        assert rc == hc.HC_ERR_STATE
        t = srv.submit(0, q[:2000], 10, 2000)
        first = srv.poll(t, 0)                    # may or may not be done yet
        if first is None:
            assert srv.poll(t, 30_000_000) is not None
        rc = hc.lib().hc_serve_poll(srv.handle, t, None, None, 0)
        assert rc == hc.HC_ERR_STATE              # already collected
        with pytest.raises(hc.HCError):
            srv.submit(5, q[:2], 10, 10)          # no such index
    finally:
        srv.close()


def test_destroy_with_requests_in_flight(hc, indexes):
    ix, q = indexes[0]
    srv = hc.hc_serve_create([ix], 64 << 20)
    for j in range(10):
        srv.submit(0, q[j * 100:(j + 1) * 100], 10, 300)
    srv.close()                                    # drains, then frees; must not hang


def test_create_reports_injected_oom(hc, indexes):
    ix, _ = indexes[0]
    for after in (0, 1):
        hc.hc_debug_fail_alloc(after)
        try:
            with pytest.raises(hc.HCError) as e:
                hc.hc_serve_create([ix], 1 << 20)
            assert e.value.status == hc.HC_ERR_OOM
        finally:
            hc.hc_debug_fail_alloc(-1)
    srv = hc.hc_serve_create([ix], 1 << 20)
    srv.close()

"""Host-buffer paths that overlap copies with compute: hc_build_host_async
(rows uploaded on a copy stream, the build queued behind an event) gives the
lists of hc_build, refuses pageable rows, and, pipelined two databases
ahead as the bench's end-to-end loop runs it, answers every step as the
oracle; hc_query_host answers batches of 4096 queries or more in key order
with the results of the input-order walk."""
import ctypes
import collections

import numpy as np
import pytest

from helpers import dev
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


def sync():
    import torch
    torch.cuda.synchronize()


@pytest.mark.parametrize("side_copy,parts", [(True, 1), (False, 1), (True, 3)])
def test_async_host_build_equals_device_build(hc, side_copy, parts):
    import torch
    n = 30_011
    db = datagen.make_db(n, 128, seed=31)
    pinned = torch.from_numpy(db).pin_memory()
    build_s, copy_s = torch.cuda.Stream(), torch.cuda.Stream()
    idx_a = hc.hc_build_host_async(pinned, partitions=parts, stream=build_s,
                                   copy_stream=copy_s if side_copy else None)
    idx_d = hc.hc_build(dev(db), partitions=parts)
    build_s.synchronize()
    for x, y in zip(hc.hc_index_copy_lists(idx_a)[:3], hc.hc_index_copy_lists(idx_d)[:3]):
        sync()
        assert torch.equal(x, y)
    q = datagen.make_queries(db, 150, seed=32)
    ids, dist = hc.hc_query_host(idx_a, q, 10, 40)
    oidx = O.build(db, curves=8, m=16, ell=parts)
    rids, rdist = O.search(oidx, db, q, 10, 40)
    assert np.array_equal(ids.numpy(), rids)
    assert np.array_equal(dist.numpy(), O.int32_dist(rdist))
    idx_a.free()
    idx_d.free()


def test_async_host_build_refuses_pageable_rows(hc):
    db = np.zeros((1000, 128), np.uint8)
    p, keep = hc._params(1000, 128, hc.HC_U8, 8, 16, None, 1)
    h = ctypes.c_void_p()
    rc = hc.lib().hc_build_host_async(ctypes.c_void_p(db.ctypes.data), ctypes.byref(p), None,
                                      None, ctypes.byref(h))
    assert rc == hc.HC_ERR_ARG and not h.value


def test_pipelined_steps_match_the_oracle(hc):
    """Four databases, each step's rows and queries queued two steps ahead on
    one copy stream (builds on a second stream, walks on a third), as the
    bench's end-to-end loop runs them: each step's results are the oracle's
    for its own database."""
    import torch
    n, nq, steps, depth = 12_000, 4_500, 4, 2
    dbs = [datagen.make_db(n, 128, seed=40 + i) for i in range(steps)]
    qs = [datagen.make_queries(d, nq, seed=50 + i) for i, d in enumerate(dbs)]
    pinned = [torch.from_numpy(d).pin_memory() for d in dbs]
    qpin = [torch.from_numpy(q).pin_memory() for q in qs]
    outs = [(torch.empty((nq, 10), dtype=torch.int32).pin_memory(),
             torch.empty((nq, 10), dtype=torch.int32).pin_memory()) for _ in range(steps)]
    copy_s, build_s, query_s = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    ahead = collections.deque()

    def enqueue(j):
        idx = hc.hc_build_host_async(pinned[j], stream=build_s, copy_stream=copy_s)
        built = torch.cuda.Event()
        built.record(build_s)
        query_s.wait_event(built)
        hc.hc_query_host_async(idx, qpin[j], 10, 64, outs[j][0], outs[j][1], stream=query_s,
                               copy_stream=copy_s)
        done = torch.cuda.Event()
        done.record(query_s)
        ahead.append((idx, done))

    queued = 0
    while queued < depth:
        enqueue(queued)
        queued += 1
    for i in range(steps):
        if queued < steps:
            enqueue(queued)
            queued += 1
        idx, done = ahead.popleft()
        done.synchronize()
        idx.free(stream=query_s)
        oidx = O.build(dbs[i], curves=8, m=16)
        rids, rdist = O.search(oidx, dbs[i], qs[i], 10, 64)
        assert np.array_equal(outs[i][0].numpy(), rids), i
        assert np.array_equal(outs[i][1].numpy(), O.int32_dist(rdist)), i
    sync()


def test_async_host_query_refuses_pageable_buffers(hc):
    import torch
    db = datagen.make_db(3000, 128, seed=70)
    idx = hc.hc_build(dev(db))
    q = np.ascontiguousarray(db[:10])
    ids = np.zeros((10, 10), np.int32)
    dist = np.zeros((10, 10), np.int32)
    rc = hc.lib().hc_query_host_async(idx.handle, ctypes.c_void_p(q.ctypes.data), 10, 10, 16,
                                      ctypes.c_void_p(ids.ctypes.data),
                                      ctypes.c_void_p(dist.ctypes.data), None, None)
    assert rc == hc.HC_ERR_ARG
    # the same call from pinned buffers, and a second one reusing the staging
    qp = torch.from_numpy(q).pin_memory()
    oi = torch.zeros((10, 10), dtype=torch.int32).pin_memory()
    od = torch.zeros((10, 10), dtype=torch.int32).pin_memory()
    for _ in range(2):
        hc.hc_query_host_async(idx, qp, 10, 16, oi, od)
        sync()
        ids_d, dist_d = hc.hc_query(idx, dev(q), 10, 16)
        sync()
        assert torch.equal(oi, ids_d.cpu()) and torch.equal(od, dist_d.cpu())
    idx.free()


def test_large_host_batches_in_key_order(hc):
    import torch
    n = 20_000
    db = datagen.make_db(n, 128, seed=61)
    idx = hc.hc_build(dev(db))
    for nq in (4095, 4096, 10_001):
        q = datagen.make_queries(db, nq, seed=nq)
        ids_h, dist_h = hc.hc_query_host(idx, q, 10, 48)
        ids_d, dist_d = hc.hc_query(idx, dev(q), 10, 48)
        sync()
        assert torch.equal(ids_h, ids_d.cpu()) and torch.equal(dist_h, dist_d.cpu()), nq
    q = datagen.make_queries(db, 5000, seed=7)
    ids_h, dist_h = hc.hc_query_host(idx, q, 10, 48)
    oidx = O.build(db, curves=8, m=16)
    rids, rdist = O.search(oidx, db, q, 10, 48)
    assert np.array_equal(ids_h.numpy(), rids)
    assert np.array_equal(dist_h.numpy(), O.int32_dist(rdist))
    idx.free()

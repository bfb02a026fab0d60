"""Parity at the benchmark's full size, in the launch configuration bench.py
times: N = 10,000,000 uint8 rows of 128 dims, 8 curves of 16 dims, one query
launch of Q = 100,000 queries, k = 10.

The oracle builds its own index over all 10M rows (Algorithm 1, ~10 s on the
host cores); every one of the 80M list entries must match the GPU's, and a
seeded sample of the queries is searched by the oracle one by one and must
match the GPU's full-batch results bit for bit (ids and int32 distances), at
p = 32, 128 and 512, through hc_query and through hc_query_ordered (the
bench's launch sequence), and with 8 and 32 partitions.  The float32 variant
(x = u/255) is checked the same way on a sample, within 1e-5 relative.
"""
import numpy as np
import pytest

from helpers import compare_f32, u64
from oracle import oracle as O
from paper_1209_0410_gb300 import datagen

pytestmark = pytest.mark.gpu

N, Q, K = 10_000_000, 100_000, 10
SAMPLE = 400


@pytest.fixture(scope="module")
def hc():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1209_0410_gb300 import hc as _hc
    _hc.lib()
    return _hc


@pytest.fixture(scope="module")
def data():
    db = datagen.make_db(N, 128, seed=datagen.SEED_DB)
    q = datagen.make_queries(db, Q, seed=datagen.SEED_QUERIES)
    pick = np.sort(np.random.default_rng(2024).choice(Q, size=SAMPLE, replace=False))
    return db, q, pick


@pytest.fixture(scope="module")
def oracle_index(data):
    db, _, _ = data
    return O.build(db, curves=8, m=16)


@pytest.fixture(scope="module")
def gpu_index(hc, data):
    import torch
    db, _, _ = data
    tdb = torch.from_numpy(db).cuda()
    idx = hc.hc_build(tdb, 8, 16)
    torch.cuda.synchronize()
    yield idx
    idx.free()


def test_full_size_lists_bit_exact(hc, gpu_index, oracle_index):
    import torch
    hi, lo, ids, off = hc.hc_index_copy_lists(gpu_index)
    torch.cuda.synchronize()
    assert np.array_equal(off, oracle_index.list_off)
    assert np.array_equal(u64(hi), oracle_index.keys_hi)
    assert np.array_equal(u64(lo), oracle_index.keys_lo)
    assert np.array_equal(ids.cpu().numpy().view(np.uint32), oracle_index.ids)


@pytest.mark.parametrize("p", [128, 32, 512])
def test_full_batch_query_sampled_bit_exact(hc, data, gpu_index, oracle_index, p):
    import torch
    db, q, pick = data
    ids, dist = hc.hc_query(gpu_index, torch.from_numpy(q).cuda(), K, p)
    torch.cuda.synchronize()
    rids, rdist = O.search(oracle_index, db, q[pick], K, p)
    assert np.array_equal(ids.cpu().numpy()[pick], rids)
    assert np.array_equal(dist.cpu().numpy()[pick], O.int32_dist(rdist))


def test_full_batch_ordered_query_sampled_bit_exact(hc, data, gpu_index, oracle_index):
    """The launch sequence bench.py times: hc_query_ordered (order keys of
    every curve, the batch lower_bound pass over the fence, the walk in
    curve-0 key order) over the whole batch at p = 128."""
    import torch
    db, q, pick = data
    ids, dist = hc.hc_query_ordered(gpu_index, torch.from_numpy(q).cuda(), K, 128)
    torch.cuda.synchronize()
    rids, rdist = O.search(oracle_index, db, q[pick], K, 128)
    assert np.array_equal(ids.cpu().numpy()[pick], rids)
    assert np.array_equal(dist.cpu().numpy()[pick], O.int32_dist(rdist))


@pytest.mark.parametrize("ell,phi", [(32, 4), (8, 32)])
def test_full_size_partitioned_ordered_sampled(hc, data, ell, phi):
    """Partitioned Hypercurves at full size (256 and 64 lists of 0.3M and
    1.25M entries): the ordered path's batch search and walk against the
    oracle's partitioned Algorithm 2 on the sampled queries."""
    import torch
    db, q, pick = data
    idx = hc.hc_build(torch.from_numpy(db).cuda(), 8, 16, partitions=ell)
    ids, dist = hc.hc_query_ordered(idx, torch.from_numpy(q).cuda(), K, phi)
    torch.cuda.synchronize()
    idx.free()
    oidx = O.build(db, curves=8, m=16, ell=ell)
    rids, rdist = O.search(oidx, db, q[pick], K, phi)
    assert np.array_equal(ids.cpu().numpy()[pick], rids)
    assert np.array_equal(dist.cpu().numpy()[pick], O.int32_dist(rdist))


def test_full_size_float32_sampled(hc, data):
    import torch
    db, q, pick = data
    dbf, qf = datagen.to_f32(db), datagen.to_f32(q)
    idx = hc.hc_build(torch.from_numpy(dbf).cuda(), 8, 16)
    ids, dist = hc.hc_query(idx, torch.from_numpy(qf).cuda(), K, 128)
    torch.cuda.synchronize()
    oidx = O.build(dbf, curves=8, m=16)
    rids, rdist = O.search(oidx, dbf, qf[pick], K, 128)
    probs = compare_f32(ids.cpu().numpy()[pick], dist.cpu().numpy()[pick], rids, rdist)
    assert not probs, probs[:5]
    idx.free()
